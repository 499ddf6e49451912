// smf_residue_gemm_noalloc: the residue product without any allocation.
//
// Some callers cannot call cudaMalloc: code that runs while another component
// owns the device allocator (a framework's caching pool, a memory-capped
// process), code on a latency-critical path where an allocation's implicit
// device synchronisation is not acceptable, and plugins that are handed only
// input and output buffers.  For them this entry point takes its scratch -
// the bf16 digit planes of both operands that the tensor-core product reads -
// from one file-scope device array of fixed size instead of a workspace.
//
// The array lives in this file; host code only ever sees its host-side
// stand-in, so the device address is looked up with cudaGetSymbolAddress with
// the device current.  The address belongs to the device's current context:
// it is cached per device together with that context's handle and looked up
// again when the context has changed (after cudaDeviceReset, or when the
// primary context was released and created anew).
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "smf_internal.h"

namespace {

// Fixed scratch: 64 MiB, held by every GPU that loads this library until the
// process exits.
constexpr size_t kNoallocScratchBytes = 64ull << 20;
static __device__ __align__(256) uint8_t g_noalloc_scratch[kNoallocScratchBytes];

constexpr int kMaxDevices = 256;
std::mutex g_noalloc_mu;
struct ScratchAddr {
    CUcontext ctx;
    void* addr;
};
ScratchAddr g_noalloc_addr[kMaxDevices] = {};

// The current context's handle through the driver entry point (the library
// links only the CUDA runtime).
CUcontext current_context() {
    using Fn = CUresult (*)(CUcontext*);
    static Fn fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return (Fn)p;
    }();
    CUcontext c = nullptr;
    if (!fn || fn(&c) != CUDA_SUCCESS) return nullptr;
    return c;
}

// Device address of the scratch array on `device` (which must be current).
int noalloc_scratch(int device, void** out, std::string* err) {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (device < 0 || device >= kMaxDevices) {
        *err = "noalloc: device index out of range";
        return SMF_E_INVALID;
    }
    const CUcontext cur = current_context();
    ScratchAddr& e = g_noalloc_addr[device];
    if (!e.addr || !cur || e.ctx != cur) {
        void* p = nullptr;
        const cudaError_t rc = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (rc != cudaSuccess || !p) {
            *err = std::string("noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(rc);
            return SMF_E_CUDA;
        }
        e.addr = p;
        e.ctx = cur;
    }
    *out = e.addr;
    return SMF_OK;
}

struct CurrentDevice {
    int prev = -1;
    explicit CurrentDevice(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~CurrentDevice() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

int noalloc_fail(smf_ctx* ctx, int code, const std::string& msg) {
    ctx->err = msg;
    return code;
}

}  // namespace

extern "C" int smf_residue_gemm_noalloc(smf_ctx* ctx, const smf_basis* b, const int32_t* A,
                                        int64_t a_prime_stride, const int32_t* B, int32_t* C, int64_t M,
                                        int64_t N, int64_t K, void* stream) {
    using namespace smf;
    if (!ctx || !b) return SMF_E_INVALID;
    if (ctx->form != SMF_FORM_INT8LIMB)  // the FP64 form needs no scratch at all
        return smf_residue_gemm(ctx, b, A, a_prime_stride, B, C, M, N, K, nullptr, 0, stream);
    if (M < 0 || N < 0 || K < 0 || a_prime_stride < 0)
        return noalloc_fail(ctx, SMF_E_INVALID, "residue_gemm_noalloc: bad sizes");
    if (a_prime_stride != 0 && a_prime_stride < M * K)
        return noalloc_fail(ctx, SMF_E_INVALID, "residue_gemm_noalloc: a_prime_stride overlaps");
    if (M * N > 0 && (!C || (K > 0 && (!A || !B))))
        return noalloc_fail(ctx, SMF_E_INVALID, "residue_gemm_noalloc: null operand");
    const int L = (int)b->primes.size();
    const bool shared = a_prime_stride == 0;
    const uint64_t amax = (shared ? b->primes.back() : b->primes[0]) / 2, bmax = b->primes[0] / 2;
    const int TA = digits_for(amax), TB = digits_for(bmax);
    if (TA > 3 || TB > 3) return noalloc_fail(ctx, SMF_E_UNSUPPORTED, "residue_gemm_noalloc: more than 3 digits");
    if ((unsigned __int128)K * amax * bmax >= ((unsigned __int128)1 << 62))
        return noalloc_fail(ctx, SMF_E_UNSUPPORTED, "residue_gemm_noalloc: K * |a| * |b| must stay below 2^62");
    // scratch layout: A digit planes, then B digit planes (256-byte aligned)
    const int64_t ld = round_up(K > 0 ? K : 1, 8);
    const size_t a_bytes = (size_t)TA * (shared ? 1 : L) * M * ld * 2;
    const size_t b_off = (a_bytes + 255) / 256 * 256;
    const size_t need = b_off + (size_t)TB * L * N * ld * 2;
    if (need > kNoallocScratchBytes)
        return noalloc_fail(ctx, SMF_E_NOMEM,
                            "residue_gemm_noalloc: this product needs " + std::to_string(need) +
                                " bytes of scratch; the fixed scratch holds " +
                                std::to_string(kNoallocScratchBytes));
    CurrentDevice cd(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (M * N == 0) return SMF_OK;
    cudaError_t e;
    if (K == 0) {  // empty inner dimension: every residue is 0
        e = cudaMemsetAsync(C, 0, sizeof(int32_t) * (size_t)L * M * N, s);
        return e == cudaSuccess ? SMF_OK : noalloc_fail(ctx, SMF_E_CUDA, cudaGetErrorString(e));
    }
    void* scratch = nullptr;
    std::string err;
    const int st = noalloc_scratch(ctx->device, &scratch, &err);
    if (st != SMF_OK) return noalloc_fail(ctx, st, err);
    uint8_t* w = (uint8_t*)scratch;
    // every digit the product reads is rewritten here, so the leftovers of an
    // earlier call never need clearing
    {
        ProfScope ps(ctx, 1, s);
        e = launch_residue_digits(b->dev, A, a_prime_stride, shared ? 1 : L, M, K, w, ld, TA, false, s);
        if (e == cudaSuccess) e = launch_residue_digits(b->dev, B, K * N, L, K, N, w + b_off, ld, TB, true, s);
    }
    if (e == cudaSuccess) {
        ProfScope ps(ctx, 2, s);
        // a pending failure injection (smf_debug_inject) applies to this launch, as in smf_residue_gemm
        LimbGemmArgs la{w, ld, shared ? 1 : 0, w + b_off, ld, C, M, N, K, TA, TB, ctx->d_status, ctx->inject,
                        amax, bmax};
        ctx->inject = 0;
        e = launch_gemm_limb(ctx, b->dev, la, s);
    }
    if (e != cudaSuccess) return noalloc_fail(ctx, SMF_E_CUDA, std::string("residue_gemm_noalloc: ") + cudaGetErrorString(e));
    return SMF_OK;
}
