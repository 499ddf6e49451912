/*
 * smf.h - C ABI of the GB300 RNS exact integer matrix product.
 *
 * The library computes exact products of big-integer matrices the way the
 * Smith massager implementation does (Wang, Birmpilis, Labahn, Storjohann,
 * "A C implementation of the Smith massager algorithm", Section 3.1):
 * reduce the operands modulo a basis of word-size primes (rns_reduce),
 * multiply the residue matrices prime by prime with an exact modular product
 * (residue_gemm), and rebuild the integer result by the Chinese Remainder
 * Theorem (crt_reconstruct).  Every result is exact: there is no tolerance.
 *
 * Conventions
 *  - Every call returns an int status (SMF_OK on success).  On failure the
 *    context keeps a message readable with smf_last_error().
 *  - Ownership: the caller owns every input, output and workspace buffer.
 *    The library owns only the context, bases and the small constant tables
 *    they hold on the device.
 *  - Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy
 *    default stream).  Every call only enqueues work on that stream and
 *    returns; results are ready once the stream has been synchronised.
 *  - Big integers: W little-endian 64-bit words per entry holding the two's
 *    complement value; a matrix is row-major with leading dimension `ld`
 *    counted in entries (so entry (r, c) starts at word (r*ld + c)*W).
 *  - Residues: int32, layout [L][rows][cols] (prime-major), canonical
 *    representatives in [0, p_i) unless a call says otherwise.
 *  - Device pointers must be 16-byte aligned.
 */
#ifndef SMF_H
#define SMF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define SMF_OK 0
#define SMF_E_INVALID 1          /* bad argument, shape or layout */
#define SMF_E_SINGULAR 2         /* the matrix is singular (Smith-form driver, inverse mod p) */
#define SMF_E_NOMEM 3            /* workspace too small or allocation failed */
#define SMF_E_CUDA 4             /* a CUDA runtime/driver call failed */
#define SMF_E_BOUND 5            /* output words cannot hold the result bound */
#define SMF_E_TIMEOUT 6          /* a bounded device wait gave up */
#define SMF_E_RETRY_EXHAUSTED 7  /* the Smith-form driver's Phase 3 rejected every attempt */
#define SMF_E_UNSUPPORTED 8      /* shape or basis outside what a form handles */

/* Residue-product engine (Section 3.1 computes each residue product as an
 * exact floating-point GEMM).
 *  SMF_FORM_FP64     : residues held in fp64, exact while every partial dot
 *                      product stays below 2^53 (k-blocked), as the paper does.
 *  SMF_FORM_INT8LIMB : residues split into balanced 8-bit digits held exactly
 *                      in bf16, multiplied on the tcgen05 tensor cores with
 *                      fp32 accumulation k-blocked below 2^24, digits
 *                      recombined exactly in the epilogue.                   */
typedef enum { SMF_FORM_FP64 = 0, SMF_FORM_INT8LIMB = 1 } smf_form;

typedef struct smf_ctx smf_ctx;
typedef struct smf_basis smf_basis;

/* A big-integer matrix.  `bits` declares |x| <= 2^bits for every entry
 * (0 = derive from the word count: 64*words - 1).  The declared bound picks
 * the prime basis and, in the INT8-limb form, the digit bounds that keep the
 * tensor-core accumulation exact.  The products (smf_rns_matmul, its grouped
 * form, the server's jobs and the lifting) check every operand entry against
 * it while they reduce the operands: an entry outside [-2^bits, 2^bits] sets
 * a flag and the next smf_status_sync() returns SMF_E_BOUND (the product's
 * output is then undefined).  smf_rns_reduce and smf_inverse_mod_p reduce
 * every word exactly and do not check. */
typedef struct {
    int64_t rows, cols, ld;
    int32_t words;
    int32_t bits;
    void* data;
    int32_t on_device; /* 1: device pointer; 0: host pointer */
    int32_t reserved;
} smf_bigmat;

/* Create a context on CUDA device `device` using residue-product engine
 * `form`.  hbm_budget_bytes caps workspace the library may allocate itself
 * (0 = no cap).  Errors: SMF_E_INVALID, SMF_E_CUDA, SMF_E_UNSUPPORTED (the
 * device is not sm_103). */
int smf_create(smf_ctx** ctx, int device, smf_form form, size_t hbm_budget_bytes);

/* Destroy a context (frees library-owned device memory). NULL is a no-op. */
int smf_destroy(smf_ctx* ctx);

/* Message of the last failing call on this context ("" if none). */
const char* smf_last_error(const smf_ctx* ctx);

/* Section 3.1, basis choice: a run of consecutive primes below p_max
 * (descending, largest first) until their product M exceeds 2^(bound_bits+1),
 * so that every x with |x| <= 2^bound_bits is recovered uniquely from its
 * residues as the representative in (-M/2, M/2].  p_max = 0 picks the
 * context form's default (2^26 for FP64, 2^24 for INT8LIMB); p_max must be
 * <= 2^26.  The basis also holds, on the context's device, the constants
 * computed once for it (Section 3.1): reciprocals, Barrett and Shoup
 * factors, and the Garner inverses.
 * Errors: SMF_E_INVALID. */
int smf_basis_create(smf_ctx* ctx, int32_t bound_bits, uint32_t p_max, smf_basis** out);

/* Free a basis.  NULL is a no-op. */
int smf_basis_destroy(smf_basis* basis);

/* Number of primes L and a pointer to them (host memory owned by the basis,
 * valid until smf_basis_destroy). */
int smf_basis_info(const smf_basis* basis, int32_t* L, const uint32_t** primes);

/* Section 3.1, reduction: residues[i][r][c] = X[r][c] mod p_i in [0, p_i)
 * for all L primes of `basis`.  X must be on the device; `residues` is a
 * device buffer of L*rows*cols int32.  Errors: SMF_E_INVALID. */
int smf_rns_reduce(smf_ctx* ctx, const smf_basis* basis, const smf_bigmat* X,
                   int32_t* residues, void* stream);

/* Section 3.1, one exact modular product per prime:
 *   C_i = A_i * B_i mod p_i   (canonical, [L][M][N] int32, device)
 * A_i is the M x K int32 matrix at A + i*a_prime_stride (row-major); a
 * stride of 0 shares one A across all primes.  B is [L][K][N] int32.
 * Every entry of A_i, B_i must lie in (-p_i, p_i); a shared A must satisfy
 * |a| <= (p_L - 1)/2 for the smallest prime p_L.  The context's form picks
 * the engine.  `workspace` (device) must hold smf_residue_gemm_workspace()
 * bytes.  Errors: SMF_E_INVALID, SMF_E_NOMEM (workspace too small),
 * SMF_E_UNSUPPORTED (K beyond the exactness bound of the form). */
int smf_residue_gemm(smf_ctx* ctx, const smf_basis* basis, const int32_t* A,
                     int64_t a_prime_stride, const int32_t* B, int32_t* C,
                     int64_t M, int64_t N, int64_t K, void* workspace,
                     size_t workspace_bytes, void* stream);

/* smf_residue_gemm without any allocation (the paper has no counterpart:
 * this is a service for callers of this library).  Some callers cannot call
 * cudaMalloc - code running while another component owns the device
 * allocator, code that must not take an allocation's implicit device
 * synchronisation, plugins handed only their input and output buffers - and
 * cannot provide the workspace smf_residue_gemm needs.  This variant takes
 * the same arguments minus the workspace and keeps its scratch (the bf16
 * digit planes of both operands) in one fixed 64 MiB device array built into
 * the library, which every GPU that loads the library holds until the
 * process exits.  It calls no cudaMalloc, cudaFree or other allocating
 * routine.
 *  - Products whose digit planes exceed 64 MiB are rejected with
 *    SMF_E_NOMEM (smf_last_error gives the bytes needed).
 *  - The first call on a device looks up the array's device address on that
 *    device; make that first call before any stream capture.
 *  - All calls share the one array, which keeps the last call's contents:
 *    calls whose work overlaps on the GPU (different streams, or different
 *    host threads without ordering) race and give wrong results.  Every
 *    scratch byte a call reads is written by that same call first.
 *  - The FP64 form needs no scratch; for it this is smf_residue_gemm.
 * Errors: as smf_residue_gemm. */
int smf_residue_gemm_noalloc(smf_ctx* ctx, const smf_basis* basis, const int32_t* A,
                             int64_t a_prime_stride, const int32_t* B, int32_t* C,
                             int64_t M, int64_t N, int64_t K, void* stream);

/* Workspace bytes smf_residue_gemm needs for these sizes. */
int smf_residue_gemm_workspace(smf_ctx* ctx, const smf_basis* basis, int64_t M,
                               int64_t N, int64_t K, int a_shared, size_t* bytes);

/* Section 3.1, reconstruction: X[r][c] = the unique x in (-M/2, M/2] with
 * x = residues[i][r][c] (mod p_i) for every prime.  Computed in Lagrange form
 * with an fp32 estimate of the multiple of M to subtract; entries whose
 * estimate is too close to call take the exact mixed-radix (Garner) route.
 * residues: device [L][rows][cols] canonical.  X_out must be on the device,
 * rows x cols, and 64*words >= bit length of M (else SMF_E_BOUND).  Entries
 * not in [0, p_i) give undefined results. */
int smf_crt_reconstruct(smf_ctx* ctx, const smf_basis* basis, const int32_t* residues,
                        smf_bigmat* X_out, void* stream);

/* Section 3.1, conversion between RNS bases (the Lagrange shortcut with a
 * floating-point correction): given residues modulo the primes p_i of
 * `from` of integers x, taken as the symmetric representatives in
 * [-(M-1)/2, (M-1)/2] with M = prod p_i, write their residues modulo the
 * primes q_j of `to`, without reconstructing x.  With H = (M-1)/2,
 * xi_i = (r_i + H) (M/p_i)^-1 mod p_i and alpha = floor(sum_i xi_i / p_i)
 * (an fp32 estimate, settled exactly when it is too close to an integer):
 *   out_j = (sum_i xi_i (M/p_i mod q_j) - alpha (M mod q_j) - H) mod q_j.
 * residues_in: device int32 [L_from][count], canonical in [0, p_i).
 * residues_out: device int32 [L_to][count], canonical in [0, q_j).  The
 * buffers must not overlap.  Either basis may hold at most 48 primes.  A
 * target prime shared with the source basis returns that prime's residues.
 * Asynchronous on `stream`.  Errors: SMF_E_INVALID (null basis, negative
 * count, a buffer not in device memory), SMF_E_UNSUPPORTED (more than 48
 * primes).  Inputs outside [0, p_i) give undefined results. */
int smf_base_convert(smf_ctx* ctx, const smf_basis* from, const smf_basis* to,
                     const int32_t* residues_in, int32_t* residues_out, int64_t count,
                     void* stream);

/* Section 3.1, the whole RNS product: C = A * B exactly.
 * A is M x K, B is K x N, C is M x N; each may live on the host or the
 * device (host buffers are staged through the workspace: pinned host memory
 * gives asynchronous copies).  The basis covers |C| <= K 2^A.bits 2^B.bits;
 * SMF_E_BOUND if C.words cannot hold that bound.  `workspace` (device) must
 * hold smf_rns_matmul_workspace() bytes; NULL lets the context allocate
 * (and cache) it, which may synchronise the device.
 * With A or C in host memory and M > 1024 the product runs as row chunks:
 * the host copies go through the context's own copy-in and copy-out streams
 * and overlap the other chunks' kernels.  They start after the work already
 * queued on `stream`, and later work on `stream` starts after them, so the
 * call stays ordered on `stream`.  A context runs one such call at a time
 * (its copy streams, events and staging slots are shared).
 * Errors: SMF_E_INVALID, SMF_E_BOUND, SMF_E_NOMEM, SMF_E_UNSUPPORTED. */
int smf_rns_matmul(smf_ctx* ctx, const smf_bigmat* A, const smf_bigmat* B, smf_bigmat* C,
                   void* workspace, size_t workspace_bytes, void* stream);

/* Workspace bytes smf_rns_matmul needs for these operands. */
int smf_rns_matmul_workspace(smf_ctx* ctx, const smf_bigmat* A, const smf_bigmat* B,
                             const smf_bigmat* C, size_t* bytes);

/* Section 3.1's product for a batch: C[i] = A[i] * B[i] exactly for every
 * i < count, products of any shapes.  This is what Phase 2's batches of
 * products with uneven dimensions need: one basis covers the largest product
 * bound, and in the INT8-limb form the residue products of all items run in
 * one persistent launch over all their tiles, so small products share the
 * GPU instead of each leaving most SMs idle.  All operands must be on the
 * device (SMF_E_INVALID otherwise).  `workspace` as for smf_rns_matmul, sized
 * by smf_rns_matmul_grouped_workspace().  In the FP64 form the items run one
 * after another.  Errors: as smf_rns_matmul, per item. */
int smf_rns_matmul_grouped(smf_ctx* ctx, int count, const smf_bigmat* A, const smf_bigmat* B,
                           smf_bigmat* C, void* workspace, size_t workspace_bytes, void* stream);

/* Workspace bytes smf_rns_matmul_grouped needs for these operands. */
int smf_rns_matmul_grouped_workspace(smf_ctx* ctx, int count, const smf_bigmat* A,
                                     const smf_bigmat* B, const smf_bigmat* C, size_t* bytes);

/* A grouped product prepared once and replayed (Section 3.1's product for a
 * batch, as smf_rns_matmul_grouped, for callers that run the same batch
 * shapes on the same buffers again and again with new contents, as Phase 2's
 * iterations do).  smf_group_plan_create does the host work of a grouped call
 * once - the basis, the workspace layout, the work lists and the TMA tensor
 * maps, copied to a workspace the plan owns - and captures the call's kernel
 * launches in a CUDA graph; smf_group_plan_launch replays that graph on
 * `stream` (one cudaGraphLaunch).  The plan keeps the descriptors of A, B and
 * C: each launch reads the current contents of the same device buffers and
 * writes C, bit for bit what smf_rns_matmul_grouped gives for them.  The
 * buffers must stay allocated until the plan is destroyed.  Two launches of
 * one plan that overlap on the GPU race on its workspace.  In the FP64 form,
 * or when a product falls outside the grouped kernels, a launch runs
 * smf_rns_matmul on each product in turn (no graph).
 * flags:
 *  SMF_PLAN_AUTOTUNE: choose the launch configuration by measurement.  For
 *    each class of products (basis size, A's digit count, a shared A,
 *    rounded-up log2 of K, M and N) the class's products run alone in each
 *    candidate variant: as planned; with the residue product's copy warp
 *    fetching the tiles four K steps ahead into L2; for a shared A that needs
 *    fewer than three digits, with A padded to three (zero) digits, whose tile
 *    has a faster MMA issue pattern; and for a one-digit A, in a launch of its
 *    own whose copy ring holds five one-digit K steps (the 3x3-digit kernel's
 *    three slots hold three).  The fastest is kept; the context
 *    remembers the choice per class, so later plans reuse it without
 *    measuring.  When the batch then mixes digit counts, the whole batch also
 *    runs with its tiles ordered longest K first and most MMAs per tile
 *    first, and the faster order is kept.  Every candidate is exact, so these
 *    runs write C with the correct product; they take a few launches of each
 *    class.
 *  SMF_PLAN_PAD_ALL / SMF_PLAN_PREFETCH / SMF_PLAN_ONE_DIGIT /
 *    SMF_PLAN_ORDER_WORK (without SMF_PLAN_AUTOTUNE): fix those choices
 *    instead (padding for every narrow shared A; the L2 prefetch for every
 *    product; the one-digit kernel for every one-digit A not padded;
 *    MMA-work order).
 * Operands must be on the device.  create is synchronous on `stream`.
 * Errors: as smf_rns_matmul_grouped, SMF_E_NOMEM (the plan's workspace),
 * SMF_E_CUDA (capture). */
typedef struct smf_group_plan smf_group_plan;
#define SMF_PLAN_AUTOTUNE 1
#define SMF_PLAN_PAD_ALL 2
#define SMF_PLAN_ORDER_WORK 4
#define SMF_PLAN_PREFETCH 8
#define SMF_PLAN_ONE_DIGIT 16
int smf_group_plan_create(smf_ctx* ctx, int count, const smf_bigmat* A, const smf_bigmat* B, smf_bigmat* C,
                          int flags, smf_group_plan** out, void* stream);
int smf_group_plan_launch(smf_group_plan* plan, void* stream);
/* What the plan chose: graph (1: replayed as a CUDA graph), padded (products
 * whose A takes three digits instead of fewer), prefetched (products whose
 * tiles are fetched into L2 ahead of their loads), one_digit (products in the
 * one-digit kernel's launch), tile_order (0: longest K
 * first, 1: most MMAs first), classes the autotuner measured and classes it
 * took from the context's record, its time in ms, the workspace bytes.  Any
 * pointer may be NULL. */
int smf_group_plan_info(const smf_group_plan* plan, int32_t* graph, int32_t* padded, int32_t* prefetched,
                        int32_t* one_digit, int32_t* tile_order, int32_t* classes_tuned, int32_t* classes_cached,
                        double* tune_ms, size_t* workspace_bytes);
/* The autotuner's measurements, one line per decision, as text (cut to cap - 1
 * bytes, NUL-terminated; empty without SMF_PLAN_AUTOTUNE). */
int smf_group_plan_report(const smf_group_plan* plan, char* buf, int64_t cap);
/* Free the plan (its workspace and graph; allowed after its context has been
 * destroyed).  NULL is a no-op. */
int smf_group_plan_destroy(smf_group_plan* plan);

/* Section 3.1's residue products and their CRT reconstruction in one kernel
 * (enable = 1; 0 restores the default, two kernels).  With it, smf_rns_matmul
 * on operands in device memory runs the INT8-limb residue product with the
 * reconstruction in its epilogue when the product allows it (three-digit
 * residues of at most 24 primes below 2^24, no K split, and a shared A with N
 * a multiple of 64): each block of 128 rows by 64 columns of C is
 * reconstructed by the block of threads whose residue tile, the last of the
 * block's primes to be stored, completes it, while that block's tensor cores
 * already work on its next tile.  Results are bit for bit those of the two
 * kernels.  Other products, the FP64 form and host operands keep the two
 * kernels.  Errors: SMF_E_INVALID. */
int smf_set_fused_crt(smf_ctx* ctx, int enable);

/* Synchronise `stream`, then report whether any kernel of this context gave
 * up a bounded device wait since the last call (SMF_E_TIMEOUT; the flag is
 * cleared).  Kernels never spin without limit: a wait that exceeds about two
 * seconds records the timeout and the kernel returns. */
int smf_status_sync(smf_ctx* ctx, void* stream);

/* Failure injection for testing the bounded waits (no GPU fault involved).
 * SMF_INJECT_STALL_LOADS makes the next INT8-limb residue product on this
 * context launch with its copy-issuing warp idle, so the tensor-core and drain
 * warps wait on data that never arrives; each wait gives up after about two
 * seconds, the kernel unwinds (freeing its tensor memory) and the next
 * smf_status_sync() returns SMF_E_TIMEOUT.  The flag clears after one launch;
 * the results of that launch are undefined. */
#define SMF_INJECT_STALL_LOADS 1
/* SMF_INJECT_WRONG_SMITH makes the next smf_smith_form hand Phase 3 a wrong
 * candidate (its largest invariant factor doubled) in its first attempt, so
 * that Phase 3 must reject it and the call restart; with
 * SMF_INJECT_WRONG_SMITH_ALWAYS every attempt of the next call gets one and
 * the call ends with SMF_E_RETRY_EXHAUSTED.  Host-side only: no device work
 * is disturbed. */
#define SMF_INJECT_WRONG_SMITH 2
#define SMF_INJECT_WRONG_SMITH_ALWAYS 4
int smf_debug_inject(smf_ctx* ctx, int flags);

/* Kernel timing: when enabled, the library brackets each kernel it launches
 * with CUDA events on the launching stream.  smf_profile_read() synchronises
 * the events recorded since the last read and returns, per kernel kind, the
 * launch count and total milliseconds.  Kinds: 0 reduce, 1 limb/operand
 * split, 2 residue GEMM, 3 CRT, 4 host<->device staging copies. */
#define SMF_PROF_KINDS 5
int smf_profile_enable(smf_ctx* ctx, int enable);
int smf_profile_read(smf_ctx* ctx, int32_t counts[SMF_PROF_KINDS], double ms[SMF_PROF_KINDS]);

/* The FP64 form's roofline (Section 3.1 runs each residue product as an
 * exact double-precision GEMM): the measured throughput of the device's FP64
 * FMA pipe in TFLOP/s, from a kernel of independent register-resident fma
 * chains on every SM, timed with CUDA events on `stream` (best of three
 * launches after one warm-up).  Synchronous.  Errors: SMF_E_INVALID,
 * SMF_E_CUDA. */
int smf_fp64_peak(smf_ctx* ctx, double* tflops, void* stream);

/* Library version string. */
const char* smf_version(void);

/* p-adic (Dixon) lifting, the solve behind the integrality certification of
 * the paper's Phase 2 and its initialization with A^-1 mod p (Sections 2
 * and 3): for a nonsingular A (n x n) and B (n x m), with C = A^-1 mod p for
 * the one prime p of `p_basis`, run `steps` steps of
 *   X_i = C R_i mod p,   R_(i+1) = (R_i - A X_i) / p   (R_0 = B, exact),
 * so that A (sum_(i<steps) X_i p^i) + p^steps R_steps = B.  Each step is a
 * residue product with one prime and an exact product, in the context's form.
 * A and B: device, single-word entries with declared bounds (bits) such that
 * bits(A) + bits(p) + ceil(log2 n) + 2 <= 62 and bits(B) <= 61 (else
 * SMF_E_BOUND).  A_inv_mod_p: device int32 [n][n] canonical.  X_digits:
 * device int32 [steps][n][m], canonical digits.  R: device n x m single
 * words, receives R_steps (may alias B).  `workspace` holds
 * smf_padic_lift_workspace() bytes (NULL: the context allocates).  A
 * non-zero remainder in a division (A_inv_mod_p not the inverse) is reported
 * by smf_status_sync as SMF_E_INVALID.  Errors: SMF_E_INVALID, SMF_E_BOUND,
 * SMF_E_NOMEM. */
int smf_padic_lift_workspace(smf_ctx* ctx, const smf_basis* p_basis, const smf_bigmat* A, const smf_bigmat* B,
                             size_t* bytes);
int smf_padic_lift(smf_ctx* ctx, const smf_basis* p_basis, const smf_bigmat* A, const int32_t* A_inv_mod_p,
                   const smf_bigmat* B, int32_t steps, int32_t* X_digits, smf_bigmat* R, void* workspace,
                   size_t workspace_bytes, void* stream);

/* A^-1 mod p for the one prime p of `p_basis` (the initialization of the
 * p-adic lifting, Section 3): Gauss-Jordan elimination over GF(p) on the
 * device, one pivot launch and one elimination launch per column.  A: device,
 * n x n, any word count.  A_inv: device int32 [n][n], canonical residues.
 * `workspace` holds smf_inverse_mod_p_workspace(n) bytes (NULL: the context
 * allocates).  Asynchronous on `stream`; when p divides det A (a column
 * without a pivot) A_inv is undefined and the next smf_status_sync returns
 * SMF_E_SINGULAR.  Errors: SMF_E_INVALID, SMF_E_NOMEM, SMF_E_CUDA. */
int smf_inverse_mod_p_workspace(smf_ctx* ctx, int64_t n, size_t* bytes);
int smf_inverse_mod_p(smf_ctx* ctx, const smf_basis* p_basis, const smf_bigmat* A, int32_t* A_inv, void* workspace,
                      size_t workspace_bytes, void* stream);

/* Largest invariant factor s_n of a nonsingular A (the paper's Phase 1,
 * Section 2; Monte Carlo).  A: n x n single words (host or device) with
 * bits(A) + ceil(log2 n) <= 55 (else SMF_E_BOUND).  The call takes a prime
 * p < 2^b, b = min(24, 60 - bits(A) - ceil(log2 n)) (the lifting's residuals
 * stay within 64-bit words), with p not dividing det A (smf_inverse_mod_p; up
 * to 8 primes, then SMF_E_SINGULAR), lifts A^-1 B mod p^k for m random columns B
 * (|b| <= 2^10, drawn from `seed`), reconstructs a random weighted sum of each
 * column's solution as a fraction, and returns s = lcm of the m denominators.
 * The lifting stops once every column's fraction has come back unchanged at
 * two checkpoints with 64 bits of p^k to spare, and at the latest when p^k is
 * above twice the product of Hadamard's bounds.  s divides s_n and equals it
 * except with probability about (3/4)^m.
 * s_limbs: host, s_cap little-endian 32-bit limbs; *s_len gets the limb
 * count (SMF_E_NOMEM when above s_cap).  seconds (host, 4 or NULL): A^-1 mod
 * p, lifting, reconstruction, total.  Synchronous on `stream`.  Errors:
 * SMF_E_INVALID, SMF_E_SINGULAR, SMF_E_BOUND, SMF_E_NOMEM, SMF_E_CUDA. */
int smf_largest_invariant_factor(smf_ctx* ctx, const smf_bigmat* A, int32_t m, uint64_t seed, uint32_t* s_limbs,
                                 int32_t s_cap, int32_t* s_len, double seconds[4], void* stream);

/* The Smith form (Sections 1 and 2): for a nonsingular A (n x n, single-word
 * entries, host or device, |a| <= 2^A.bits with bits(A) + ceil(log2 n) <= 55,
 * n < 16384) the invariant factors s_1 | s_2 | ... | s_n, s_i > 0,
 * of the unique S = diag(s_i) = U A V with U, V unimodular.  The paper's
 * three phases, on this library's device calls and host big integers:
 *  Phase 1: s = s_n by smf_largest_invariant_factor's lifting (m = 32
 *    columns); the same lifting keeps the digits of the projection
 *    P = Q A^-1 J of A^-1 by 32 random functionals Q and 32 columns J.
 *  Phase 2: the Smith form of Rem(s P, s) over Z/(s) (a 16 x 16 corner of
 *    P first, grown to at most 32 x 32 when it holds too few), with the
 *    working modulus divided by each step's content, gives the largest
 *    invariant factors; those above 2^62 are kept, and the last iteration takes all the
 *    others at once as the Smith form of A over Z/(s'), s' < 2^62 the largest
 *    of them: elimination on the device, one prime power of s' at a time
 *    (smf_smith_local).
 *  Phase 3: prod s_i = +-det A (one sign) modulo four random primes in
 *    (2^30, 2^31), the four determinants by one elimination on the device
 *    (smf_det_mod);
 *    on a mismatch everything restarts from Phase 1 with new random choices,
 *    at most 4 attempts (then SMF_E_RETRY_EXHAUSTED).  Every candidate value
 *    divides the true invariant factor in its place, so a wrong candidate
 *    has a smaller product; it passes only if each prime divides
 *    |det A| / prod s_i -+ 1 (probability below 2^-40 for |det A| < 2^(2^20)),
 *    where the paper's Phase 3 certifies deterministically.
 * Output (host): s_(i+1) as little-endian 32-bit limbs at
 * limbs[offsets[i] .. offsets[i+1]) for i < n (offsets: n + 1 entries; a
 * value 1 has one limb).  When cap is below offsets[n] the call returns
 * SMF_E_NOMEM with offsets filled.  seconds (4 or NULL): Phase 1, Phase 2,
 * Phase 3, total, summed over the attempts; *attempts (or NULL): the attempts
 * run.  `seed` fixes every random choice.  Synchronous on `stream`.
 * Errors: SMF_E_INVALID, SMF_E_SINGULAR (det A = 0), SMF_E_BOUND,
 * SMF_E_NOMEM, SMF_E_CUDA, SMF_E_RETRY_EXHAUSTED, SMF_E_UNSUPPORTED (more
 * than 23 invariant factors above 2^62). */
int smf_smith_form(smf_ctx* ctx, const smf_bigmat* A, uint64_t seed, uint32_t* limbs, int64_t cap,
                   int64_t* offsets, double seconds[4], int32_t* attempts, void* stream);

/* det A mod q_i for count primes q_i < 2^62 (Section 2: the invariant
 * factors multiply to |det A|; Phase 3 of smf_smith_form checks that modulo
 * primes).  Gaussian elimination over GF(q) on the device, up to four primes
 * in lockstep in one column loop (each entry holds its residues side by
 * side): column k's pivot is the first unused row nonzero modulo every
 * prime, every other unused row subtracts its multiple; det = sign of the
 * pivot permutation times the pivots.  A column with no such row sends the
 * call back to one prime at a time.  Large matrices of 31-bit primes run by
 * panels of 16 columns (smf_set_elim_panels), with the same pivots.
 * A: square, single-word entries, host or device.  det: host, count values
 * in [0, q_i).  Synchronous; allocates its
 * scratch (about n^2 (4 or 8) bytes per prime).  Errors: SMF_E_INVALID (a q_i
 * not a prime below 2^62, count outside 1..64), SMF_E_NOMEM, SMF_E_CUDA. */
int smf_det_mod(smf_ctx* ctx, const smf_bigmat* A, const uint64_t* q, int32_t count, uint64_t* det, void* stream);

/* Local Smith forms of A at count distinct primes (the last iteration of
 * Phase 2 works over Z/(s') one prime power of s' at a time, Section 2): for
 * each i, counts gets e_i + 1 values, c[t] = the number of invariant factors
 * of A divisible by q_i^t for t = 0 .. e_i (c[0] = n; an invariant factor that
 * is 0 modulo q_i^e_i counts for every t), the lists one after another.
 * Elimination on the device: one joint column loop over all prime powers with
 * pivots that are units modulo every q_i, then per prime the block of unused
 * rows and deferred columns left: elimination over Z/(q^e) with unit pivots,
 * whose leftover block is divisible by q, is divided by q and is reduced
 * again over Z/(q^(e-1)).  Large matrices whose prime powers are below 2^31
 * run by panels of 16 columns (smf_set_elim_panels), with the same pivots.
 * A: square, single-word entries, host or device.
 * q_i^e_i < 2^62, count <= 16.  Synchronous.  Errors: SMF_E_INVALID,
 * SMF_E_NOMEM, SMF_E_CUDA. */
int smf_smith_local(smf_ctx* ctx, const smf_bigmat* A, const uint64_t* q, const int32_t* e, int32_t count,
                    int64_t* counts, void* stream);

/* Section 2's eliminations over Z/(m) (smf_det_mod, smf_smith_local and the
 * Phases 2 and 3 of smf_smith_form) take matrices of at least min_n columns
 * by panels of 16 columns when their entries fit 32-bit words (primes and
 * prime powers below 2^31): per column of a panel a pivot search and the
 * update of the panel alone, then the panel's pivot rows and one pass over
 * the trailing columns, which are read and written once per panel instead of
 * once per column.  Smaller matrices take one launch per column.  The pivots,
 * and so every result, are the same either way.  min_n = 0 restores the
 * defaults, 2560 for determinants and 1536 for local Smith forms (below them
 * the column loop was measured faster); it applies to later calls on this
 * context.  Errors: SMF_E_INVALID (no context, min_n < 0). */
int smf_set_elim_panels(smf_ctx* ctx, int64_t min_n);

/* Rational reconstruction (host only, no device work): the fraction a / b in
 * lowest terms with a = b u (mod P), |a| < 2^nb and 0 < b < 2^db, by the
 * extended Euclidean algorithm; unique when P > 2^(nb+db+1).  u and P are
 * little-endian 32-bit limbs; num and den (cap limbs each) get |a| and b,
 * *num_neg the sign of a.  Errors: SMF_E_INVALID (bad argument, or no such
 * fraction), SMF_E_NOMEM (cap too small). */
int smf_rational_reconstruct(const uint32_t* u, int32_t ulen, const uint32_t* P, int32_t plen, int64_t nb, int64_t db,
                             uint32_t* num, int32_t* num_len, int32_t* num_neg, uint32_t* den, int32_t* den_len,
                             int32_t cap);

/* Serving: continuous batching of exact products.  A server queues jobs
 * C = A B (operands on the device, owned by the caller and left untouched
 * until the job is done).  Each smf_server_step retires finished batches,
 * admits queued jobs in arrival order while their workspace fits what is left
 * of `budget_bytes` of device memory (a job that does not fit waits; later
 * jobs that fit may pass it), at most `max_batch` per step, and runs them as
 * one smf_rns_matmul_grouped call on one of the server's two streams, so
 * consecutive batches overlap on the device.  Workspaces come from the
 * stream-ordered allocator and return to it when their batch finishes.
 * The results are those of smf_rns_matmul on each job alone (bit for bit).
 * Not thread-safe: one host thread drives a server.  Errors: SMF_E_INVALID,
 * SMF_E_NOMEM (a job's workspace exceeds the budget, or the device cannot
 * supply it while nothing else runs), and those of smf_rns_matmul_grouped. */
typedef struct smf_server smf_server;
#define SMF_JOB_QUEUED 0
#define SMF_JOB_RUNNING 1
#define SMF_JOB_DONE 2
#define SMF_JOB_FAILED 3
int smf_server_create(smf_ctx* ctx, size_t budget_bytes, int max_batch, smf_server** out);
/* Queue a job; *job gets its id (0, 1, 2, ... in submission order). */
int smf_server_submit(smf_server* server, const smf_bigmat* A, const smf_bigmat* B, smf_bigmat* C,
                      int64_t* job);
/* One round of retire / admit / launch; never blocks on the device except
 * for the launch's own host staging.  *launched = jobs started. */
int smf_server_step(smf_server* server, int* launched);
/* A job's state (SMF_JOB_*), its status, and its submit / start / finish
 * times in seconds of a monotonic host clock (finish = the step that saw its
 * batch complete). */
int smf_server_job(const smf_server* server, int64_t job, int* state, int* status, double times[3]);
int smf_server_stats(const smf_server* server, int* queued, int* running_batches, size_t* bytes_in_use);
/* Step until every queued and running job is done. */
int smf_server_drain(smf_server* server);
int smf_server_destroy(smf_server* server);
/* The admission rule on its own (host only): admit[i] = 1 for queued job i
 * (arrival order, workspace bytes[i]) if it fits what is left of budget_left
 * after the jobs admitted before it, at most max_batch jobs.  Returns the
 * number admitted, or -1 for bad arguments. */
int smf_server_admit(size_t budget_left, int n, const size_t* bytes, int max_batch, int* admit);

/* Serving Smith-form jobs (the Smith form of Sections 1-2 for a stream of
 * requests): continuous batching on one GPU.  A server runs `workers` host
 * threads, each with its own context (device, form) and its own non-blocking
 * stream.  A submitted job (a host matrix, copied at submit; single-word
 * entries with a declared bound, as for smf_smith_form) waits in a queue; a
 * free worker takes the first queued job whose estimated device footprint
 * (64 n^2 bytes + 64 MiB) fits what is left of `budget_bytes` (0: no cap), so
 * a job that does not fit waits and later jobs that fit may pass it.  Jobs run
 * concurrently on the workers' streams and overlap on the GPU; each job's
 * state stays on the device for its whole run, and the driver's scratch is
 * allocated in stream order so that one job's frees do not stall another's
 * kernels.  Results are those of smf_smith_form on each job alone (bit for
 * bit: the seed fixes every random choice).  Errors: SMF_E_INVALID,
 * SMF_E_NOMEM (a job larger than the budget), SMF_E_CUDA. */
typedef struct smf_smith_server smf_smith_server;
int smf_smith_server_create(int device, smf_form form, size_t budget_bytes, int workers, smf_smith_server** out);
int smf_smith_server_submit(smf_smith_server* server, const smf_bigmat* A, uint64_t seed, int64_t* job);
/* A job's state (SMF_JOB_*), its status (that of smf_smith_form once run) and
 * its submit / start / finish times in seconds of a monotonic host clock. */
int smf_smith_server_job(smf_smith_server* server, int64_t job, int* state, int* status, double times[3]);
/* A finished job's invariant factors, laid out as smf_smith_form returns
 * them (offsets: n + 1 entries; SMF_E_NOMEM when cap is short, offsets
 * filled).  A failed job returns its status. */
int smf_smith_server_result(smf_smith_server* server, int64_t job, uint32_t* limbs, int64_t cap, int64_t* offsets);
/* A failed job's message (smf_last_error of the worker's context when the job
 * ended; empty for a job that did not fail), copied NUL-terminated into buf
 * and cut to cap - 1 bytes. */
int smf_smith_server_message(smf_smith_server* server, int64_t job, char* buf, int64_t cap);
int smf_smith_server_stats(smf_smith_server* server, int* queued, int* running, size_t* bytes_in_use);
/* Wait until every queued and running job is done. */
int smf_smith_server_drain(smf_smith_server* server);
/* Stop the workers (jobs not yet started are dropped) and free the server. */
int smf_smith_server_destroy(smf_smith_server* server);

#ifdef __cplusplus
}
#endif

#endif /* SMF_H */
