// oz2_gemm_noalloc: the emulated DGEMM with its scratch in a fixed, file-scope
// device array instead of memory the caller or the library allocates.
//
// Who needs it: a caller that must never see cudaMalloc happen on its behalf,
// for example an application that hands all device memory to its own pool
// under a hard budget and forbids other allocations, or a latency-critical loop
// that cannot pay for cudaMalloc's implicit device-wide synchronisation, but
// that also cannot carve out and pass a workspace itself.  Such a caller pays
// instead with a fixed amount of device memory on every GPU where this library
// is loaded, held until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "oz2.h"

namespace {

// The scratch every oz2_gemm_noalloc call works in (see OZ2_NOALLOC_SCRATCH_BYTES).
static __device__ __align__(256) unsigned char g_noalloc_scratch[OZ2_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once per
// device.  In host code `g_noalloc_scratch` only names a host-side stand-in, so
// the address must come from cudaGetSymbolAddress with the device current.
// cudaSetDevice first binds the device's primary context, the one the library's
// kernels run in, so the address is that context's even when the caller had
// another context current.
int scratch_for_current_device(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices || cudaSetDevice(dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return OZ2_ECUDA;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            (void)cudaGetLastError();
            return OZ2_ECUDA;
        }
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return OZ2_OK;
}

}  // namespace

extern "C" OZ2_API int oz2_gemm_noalloc(int m, int n, int k, const double *A, int lda, const double *B,
                                        int ldb, double *C, int ldc, int nmoduli, int mode, double target,
                                        void *stream) {
    const int nmax = nmoduli ? nmoduli : 20;
    const size_t need = oz2_workspace_size(m, n, k, nmax, mode, 0);
    if (need == 0) return OZ2_EINVAL;
    if (need > size_t(OZ2_NOALLOC_SCRATCH_BYTES)) return OZ2_ENOMEM;   // problem too large for the scratch
    void *scratch = nullptr;
    int rc = scratch_for_current_device(&scratch);
    if (rc) return rc;
    oz2_opts o = {};
    o.stream = stream;
    o.workspace = scratch;
    o.workspace_bytes = size_t(OZ2_NOALLOC_SCRATCH_BYTES);
    o.target = target;
    o.nmax = nmoduli ? 0 : nmax;
    return oz2_gemm_ex(m, n, k, A, lda, B, ldb, C, ldc, nmoduli, mode, &o);
}
