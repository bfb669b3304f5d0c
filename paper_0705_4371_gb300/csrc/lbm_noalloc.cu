// lbm_noalloc.cu -- lb_select_only_noalloc: the selection of the k largest
// values above a threshold, for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: hosts whose own allocator has reserved
// the device memory and hands it out itself, and real-time loops that must
// not take cudaMalloc's implicit device synchronisation or its latency.
// This entry point allocates nothing.  Its working memory is the fixed
// file-scope device array below; the caller passes the input values and the
// output index and count buffers, all in device memory.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/lbm.h"
#include "lbm_device.cuh"
#include "lbm_internal.h"

using namespace lbm;

namespace {

constexpr int kMaxDevices = 64;

// Working memory: candidate keys and site indices (one slot per input value)
// and the counters the kernels update.
struct NoAllocScratch {
    unsigned long long key[LB_NOALLOC_MAX_N];
    unsigned idx[LB_NOALLOC_MAX_N];
    unsigned cand_count;
    unsigned err;
    long long step;
};

// Every GPU that loads the library holds this array until the process exits.
// In host code this name is only a stand-in for the device symbol; the
// device address is obtained with cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoAllocScratch)];

std::mutex g_setup_mutex;
NoAllocScratch* g_scratch_ptr[kMaxDevices] = {};

// Failures are reported through lb_last_error, like every other entry point.
int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    set_last_error(buf);
    return code;
}

// Once per device, with that device current: the device address of the
// working memory, and the shared-memory limit of the select kernel.
int scratch_for_current_device(NoAllocScratch** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(LB_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(LB_ERR_ARG, "device index %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess)
            return fail(LB_ERR_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        e = launchers_f64(LB_D1Q3, LB_EQ_POLY).set_smem(kSelectStageCap);
        if (e != cudaSuccess)
            return fail(LB_ERR_CUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
        g_scratch_ptr[dev] = static_cast<NoAllocScratch*>(p);
    }
    *out = g_scratch_ptr[dev];
    return LB_OK;
}

}  // namespace

extern "C" int lb_select_only_noalloc(const double* ds, int n, double delta, int k, int* idx_out,
                                      int* count, void* cuda_stream) {
    if (n < 0 || k < 0) return fail(LB_ERR_ARG, "n and k must be >= 0");
    if (!count || (n > 0 && !ds) || (n > 0 && k > 0 && !idx_out))
        return fail(LB_ERR_ARG, "NULL device pointer");
    if (n > LB_NOALLOC_MAX_N)
        return fail(LB_ERR_ARG, "n = %d exceeds the fixed working memory of %d values", n,
                    LB_NOALLOC_MAX_N);
    if (delta != delta) return fail(LB_ERR_ARG, "delta is NaN");
    NoAllocScratch* s = nullptr;
    int rc = scratch_for_current_device(&s);
    if (rc != LB_OK) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e;
    if (n == 0 || k == 0) {
        e = cudaMemsetAsync(count, 0, sizeof(int), st);
        if (e != cudaSuccess) return fail(LB_ERR_CUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
        return LB_OK;
    }
    // The array keeps the previous call's contents: the counters start at zero.
    e = cudaMemsetAsync(&s->cand_count, 0,
                        sizeof(NoAllocScratch) - offsetof(NoAllocScratch, cand_count), st);
    if (e != cudaSuccess) return fail(LB_ERR_CUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
    Params P;
    memset(&P, 0, sizeof(P));
    P.nx = n; P.ny = 1; P.nxp = n; P.plane = n;
    P.delta = delta; P.deltaf = (float)delta; P.k = k;
    P.cand_key = s->key; P.cand_idx = s->idx; P.cand_count = &s->cand_count;
    P.cand_per_block = k < 1024 ? k : 1024;
    P.sel_idx = idx_out; P.sel_count = count;
    P.step = &s->step; P.err = &s->err; P.ring_cap = 1;
    e = launch_emit_from_ds(P, ds, n, st);
    if (e == cudaSuccess) e = launchers_f64(LB_D1Q3, LB_EQ_POLY).select(P, kSelectStageCap, 1, st);
    if (e != cudaSuccess) return fail(LB_ERR_CUDA, "launch: %s", cudaGetErrorString(e));
    return LB_OK;
}
