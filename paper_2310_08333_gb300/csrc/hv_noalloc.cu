// Hessian-vector product entry point that allocates no device memory.
//
// genios_op_hv needs scratch for the per-CTA partial sums of the fused rowpass, which its
// caller provides.  Some callers cannot provide it: code embedded in a host application that
// owns every byte of device memory (a serving process or plugin whose host forbids raw
// cudaMalloc and hands out no workspace), or code on a path where an allocation could fail or
// stall.  For them this variant keeps the scratch in a fixed, file-scope device array that is
// part of the library's image: it exists on every GPU that loads the library and is held until
// the process exits.
//
// Host code cannot use the array's name as a device address (on the host it only names a
// stand-in object), so the device address is looked up with cudaGetSymbolAddress once per
// device, with that device current, on the first call made on it.  Make that first call before
// any stream capture.  All calls share the array: two calls whose kernels overlap on the GPU
// (different streams, or different host threads on one device without ordering) race on it.
// Nothing in the array needs to start at zero: every CTA overwrites its whole partial row.
//
// The cached addresses belong to the device's current (primary) context.  A device reset after
// the first call (cudaDeviceReset) unloads the library's device image, and the cache then holds
// stale addresses: a process that resets a device must not call this entry point on it again.
//
// A bounded wait of the row pass that runs out (about 2 s without progress) is recorded in the
// device's op-level fault word, like genios_op_hv's: genios_op_status(stream) reports it.
#include "common.cuh"
#include "internal.h"
#include "genios.h"

#include <mutex>
#include <string>

namespace {

constexpr size_t kScratchBytes = GENIOS_HV_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_hv_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_dev_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up on first use).
cudaError_t scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_dev_addr[dev] == nullptr) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_hv_scratch);
        if (e != cudaSuccess) return e;
        g_dev_addr[dev] = p;
    }
    *out = g_dev_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" genios_status genios_op_hv_noalloc(int precision, int64_t m, int64_t n, const void* A,
                                              int64_t lda, const float* row_scale, const void* d,
                                              double nu, const void* v, void* y, void* stream) {
    using namespace genios;
    if (precision < 0 || precision > 3 || m < 1 || n < 1 || !A || !v || !y) return GENIOS_EINVAL;
    if (precision == GENIOS_FP8_E4M3 && !row_scale) return GENIOS_EINVAL;
    const int P = precision == 0 ? P_FP64 : precision == 1 ? P_FP32 : precision == 2 ? P_BF16 : P_FP8;
    RowpassPlan plan = rowpass_plan(P, m, n, lda);
    if (!plan.ok) return GENIOS_EUNSUPPORTED;
    const size_t vt = precision == 0 ? 8 : 4;
    const size_t need = (size_t)plan.grid * (size_t)lda * vt;
    if (need > kScratchBytes) {
        set_last_error("genios_op_hv_noalloc: partial sums need " + std::to_string(need) +
                       " bytes (grid x lda x value size), above the fixed " +
                       std::to_string(kScratchBytes) + "-byte scratch; use genios_op_hv with a workspace");
        return GENIOS_EINVAL;
    }
    void* scratch = nullptr;
    cudaError_t e = scratch_address(&scratch);
    if (e != cudaSuccess) {
        set_last_error(std::string("genios_op_hv_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        return GENIOS_ECUDA;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    RowpassArgs a{};
    a.prec = P;
    a.mode = RP_HV;
    a.m = m;
    a.n = n;
    a.lda = lda;
    a.A = A;
    a.row_scale = row_scale;
    a.v = v;
    a.d = d;
    a.partial = scratch;
    a.ldp = lda;
    a.wait_limit = 2000000LL * 2100LL;
    a.smem_bytes = (long long)plan.smem;
    a.partial_len = (long long)(kScratchBytes / vt);
    e = op_fault_address(&a.err);   // a bounded wait that runs out is reported by genios_op_status
    if (e != cudaSuccess) {
        set_last_error(std::string("genios_op_hv_noalloc: fault word: ") + cudaGetErrorString(e));
        return GENIOS_ECUDA;
    }
    e = rowpass_launch(a, plan, s);
    if (e == cudaSuccess) e = hv_finish(precision == 0, scratch, plan.grid, lda, n, nu, v, y, s);
    if (e != cudaSuccess) {
        set_last_error(std::string("genios_op_hv_noalloc: ") + cudaGetErrorString(e));
        return GENIOS_ECUDA;
    }
    return GENIOS_OK;
}
