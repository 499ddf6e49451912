// Internal interfaces of the Smith-form driver (Section 2's three phases):
// Phase 1's lifting run shared by smf_largest_invariant_factor and
// smf_smith_form, and the eliminations over Z/(m) of elim.cu.
#pragma once

#include <vector>

#include "bignat.h"
#include "smf_internal.h"

namespace smf {

// One run of Phase 1 (invariant.cu).  With pair_rows > 0 the run also keeps,
// per lifting digit s, the sums sum_i Q[a][i] X_s[i][j] for pair_rows random
// functionals Q (entries in [1, 2^16), drawn after the weights) and the first
// pair_cols lifted columns: sum_s (sums) p^s = Q A^-1 B (mod p^digits), the
// projection of A^-1 that Phase 2 reduces modulo s.
struct LifOptions {
    int32_t m = 32;        // random right-hand sides
    uint64_t seed = 0;
    int pair_rows = 0;     // 0, 16 or 32
    int pair_cols = 0;     // <= min(m, 32), dividing 256
    bool proven = false;   // lift to the Hadamard precision (no early stop)
};
struct LifResult {
    Nat s;                        // lcm of the denominators (divides s_n)
    uint32_t p = 0;               // the lifting prime
    int64_t digits = 0;           // p-adic digits lifted
    int64_t cap_digits = 0;       // the Hadamard precision (digits)
    std::vector<uint64_t> pair;   // [digits][pair_rows][pair_cols]
    double seconds[4] = {0, 0, 0, 0};  // A^-1 mod p, lifting, reconstruction, total
};
int lif_run(smf_ctx* ctx, const smf_bigmat* A, const LifOptions& o, LifResult* res, cudaStream_t s);

// Elimination over Z/(m) with unit pivots (elim.cu).  A: device int64,
// n x n, leading dimension lda.  det_mod_device: det A mod each of nq primes
// q_l < 2^62 (up to four at a time in one column loop).
// local_smith_device: for nq <= 16 prime powers q_l^e_l < 2^62, counts[l][t]
// (t = 0 .. e_l) = the number of invariant factors of A divisible by q_l^t
// (counts[l][0] = n): one joint column loop, then the leftover block per prime.
int det_mod_device(smf_ctx* ctx, const int64_t* A, int64_t lda, int64_t n, const uint64_t* q, int nq, uint64_t* det,
                   cudaStream_t s);
int local_smith_device(smf_ctx* ctx, const int64_t* A, int64_t lda, int64_t n, const uint64_t* q, const int* e,
                       int nq, std::vector<std::vector<int64_t>>* counts, cudaStream_t s);

}  // namespace smf
