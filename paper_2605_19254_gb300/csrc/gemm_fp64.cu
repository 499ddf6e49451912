// residue_gemm, FP64 form: the paper's own design (Section 3.1) on the GPU.
// Each residue product C_i = A_i B_i mod p_i is an fp64 GEMM whose partial
// dot products stay exact integers: the operands are centred residues, and
// after every `kblk` products the accumulators are folded with the paper's
// fast modular reduction r = a - round(a * (1/p)) * p (one fma, exact because
// a and round(a/p) * p are integers below 2^53).  The host picks kblk so that
//   |acc| <= p + kblk * amax * bmax < 2^53.
#include "smf_internal.h"

namespace smf {
namespace {

constexpr int BM = 64, BN = 64, BK = 16, TM = 4, TN = 4;  // 16 x 16 threads, 4 x 4 each

__global__ void __launch_bounds__(256)
gemm_fp64_kernel(BasisDev b, Fp64GemmArgs a, int m_tiles) {
    __shared__ double As[BK][BM + 1];
    __shared__ double Bs[BK][BN + 1];
    const int i = blockIdx.y;  // prime
    const int mt = blockIdx.x % m_tiles, nt = blockIdx.x / m_tiles;
    const int64_t m0 = (int64_t)mt * BM, n0 = (int64_t)nt * BN;
    const int32_t* Ai = a.A + (size_t)i * a.a_prime_stride;
    const int32_t* Bi = a.B + (size_t)i * a.K * a.N;
    const bool shared_a = a.a_prime_stride == 0;
    const int32_t p = (int32_t)b.p[i];
    const int32_t h = p >> 1;
    const double pd = (double)p, inv = b.inv_p[i];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;

    double acc[TM][TN];
#pragma unroll
    for (int x = 0; x < TM; x++)
#pragma unroll
        for (int y = 0; y < TN; y++) acc[x][y] = 0.0;

    int cnt = 0;
    for (int64_t k0 = 0; k0 < a.K; k0 += BK) {
        // stage A (BM x BK) and B (BK x BN) as centred fp64 residues
        for (int e = threadIdx.x; e < BM * BK; e += 256) {
            const int mm = e / BK, kk = e % BK;
            const int64_t gm = m0 + mm, gk = k0 + kk;
            int32_t v = 0;
            if (gm < a.M && gk < a.K) {
                v = Ai[gm * a.K + gk];
                if (!shared_a) {
                    if (v > h) v -= p;
                    if (v < -h) v += p;
                }
            }
            As[kk][mm] = (double)v;
        }
        for (int e = threadIdx.x; e < BK * BN; e += 256) {
            const int kk = e / BN, nn = e % BN;
            const int64_t gk = k0 + kk, gn = n0 + nn;
            int32_t v = 0;
            if (gk < a.K && gn < a.N) {
                v = Bi[gk * a.N + gn];
                if (v > h) v -= p;
                if (v < -h) v += p;
            }
            Bs[kk][nn] = (double)v;
        }
        __syncthreads();
        const int kmax = (int)(a.K - k0 < BK ? a.K - k0 : BK);
        for (int kk = 0; kk < kmax; kk++) {
            double av[TM], bv[TN];
#pragma unroll
            for (int x = 0; x < TM; x++) av[x] = As[kk][ty * TM + x];
#pragma unroll
            for (int y = 0; y < TN; y++) bv[y] = Bs[kk][tx * TN + y];
#pragma unroll
            for (int x = 0; x < TM; x++)
#pragma unroll
                for (int y = 0; y < TN; y++) acc[x][y] = fma(av[x], bv[y], acc[x][y]);
            if (++cnt == a.kblk) {  // fold: |acc| <= p afterwards
                cnt = 0;
#pragma unroll
                for (int x = 0; x < TM; x++)
#pragma unroll
                    for (int y = 0; y < TN; y++) acc[x][y] = fma(-rint(acc[x][y] * inv), pd, acc[x][y]);
            }
        }
        __syncthreads();
    }
    int32_t* Ci = a.C + (size_t)i * a.M * a.N;
#pragma unroll
    for (int x = 0; x < TM; x++) {
        const int64_t gm = m0 + ty * TM + x;
        if (gm >= a.M) continue;
#pragma unroll
        for (int y = 0; y < TN; y++) {
            const int64_t gn = n0 + tx * TN + y;
            if (gn >= a.N) continue;
            double r = fma(-floor(acc[x][y] * inv), pd, acc[x][y]);
            if (r < 0) r += pd;
            if (r >= pd) r -= pd;
            Ci[gm * a.N + gn] = (int32_t)r;
        }
    }
}

// The FP64 pipe's throughput, the roofline of the kernel above: eight
// independent fma chains per thread held in registers, on every SM.  The
// runtime operands keep the compiler from folding the chains; the result is
// stored only if it takes a value it never reaches, so nothing is written.
constexpr int kPeakChains = 8;
__global__ void __launch_bounds__(256) fp64_fma_peak_kernel(double* out, int iters, double a, double c) {
    double x[kPeakChains];
#pragma unroll
    for (int i = 0; i < kPeakChains; i++) x[i] = threadIdx.x * 1e-9 + i;
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int i = 0; i < kPeakChains; i++) x[i] = fma(x[i], a, c);
    }
    double sum = 0;
#pragma unroll
    for (int i = 0; i < kPeakChains; i++) sum += x[i];
    if (sum == -1.0) out[0] = sum;
}

}  // namespace

double fp64_fma_peak_tflops(int num_sms, cudaStream_t s) {
    const int blocks = num_sms * 8, threads = 256, iters = 8192;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 0;
    for (int rep = 0; rep < 4; rep++) {
        cudaEventRecord(e0, s);
        fp64_fma_peak_kernel<<<blocks, threads, 0, s>>>(nullptr, iters, 0.999999, 1e-7);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && (best == 0 || ms < best)) best = ms;  // the first launch warms up
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (cudaGetLastError() != cudaSuccess || best <= 0) return 0;
    const double flops = 2.0 * kPeakChains * (double)iters * blocks * threads;
    return flops / (best * 1e-3) / 1e12;
}

cudaError_t launch_gemm_fp64(const BasisDev& b, const Fp64GemmArgs& a, cudaStream_t s) {
    if (a.M == 0 || a.N == 0) return cudaSuccess;
    const int m_tiles = (int)((a.M + BM - 1) / BM);
    const int n_tiles = (int)((a.N + BN - 1) / BN);
    dim3 grid((unsigned)(m_tiles * n_tiles), (unsigned)b.L);
    gemm_fp64_kernel<<<grid, 256, 0, s>>>(b, a, m_tiles);
    return cudaGetLastError();
}

}  // namespace smf
