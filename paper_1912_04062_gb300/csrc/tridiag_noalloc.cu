// tridiag_noalloc.cu -- the symmetric tridiagonal eigensolver (bisection +
// inverse iteration on tridiag(alpha, 0, alpha)) with its scratch memory in a
// file-scope device array instead of a caller workspace, for callers that may
// not allocate device memory at all: plug-ins and libraries whose host
// application owns every device allocation (a framework's caching allocator or
// a fixed memory budget), and code that must not call cudaMalloc because it
// synchronises the device.  The paper has no counterpart; it is an interface
// convenience around the same kernels as skew_tridiag_eig.
//
// The array is SKEW_NOALLOC_SCRATCH_BYTES long and exists once per device that
// loads this library, for the life of the process.  Host code cannot use the
// array's name as a device address, so the first call on each device looks the
// address up with cudaGetSymbolAddress (with that device current) and caches
// it; later calls reuse it.  Every call shares the same array, so calls that
// overlap on the GPU (different streams, or different host threads on one
// device) race and must be serialised by the caller.
#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace sk {
namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[SKEW_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 128;
void* g_scratch_ptr[kMaxDevices] = {};
std::mutex g_scratch_mu;

// Device address of g_noalloc_scratch on the current device (looked up once).
// The address belongs to the current device only, so a stream of another
// device is refused (SKEW_ERR_UNSUPPORTED) instead of being handed an address
// it cannot use.
int scratch_address(cudaStream_t st, void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SKEW_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return SKEW_ERR_UNSUPPORTED;
    if (st) {
        int sdev = -1;
        if (cudaStreamGetDevice(st, &sdev) != cudaSuccess) {
            cudaGetLastError();
            return SKEW_ERR_CUDA;
        }
        if (sdev != dev) return SKEW_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) {
            cudaGetLastError();
            return SKEW_ERR_CUDA;
        }
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return 0;
}

}  // namespace
}  // namespace sk

using namespace sk;

extern "C" int skew_tridiag_eig_noalloc(int n, const double* alpha, int nev, double* lambda, double* Q, int ldq,
                                        int* d_status, void* stream) {
    if (n < 1) return -1;
    if (!alpha && n > 1) return -2;  // n = 1: alpha has no elements
    if (nev < 1 || nev > n) return -3;
    if (!lambda) return -4;
    if (Q && ldq < n) return -6;
    if (!d_status) return -7;
    const size_t qbytes = Q ? align_up(sizeof(double) * (size_t)n * nev) : 0;
    const size_t tbytes = tridiag_ws(n, nev);
    if (qbytes + tbytes > (size_t)SKEW_NOALLOC_SCRATCH_BYTES) return SKEW_ERR_WORKSPACE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    void* base = nullptr;
    int rc = scratch_address(st, &base);
    if (rc) return rc;
    Carve cv(base, SKEW_NOALLOC_SCRATCH_BYTES);
    double* Qi = Q ? cv.take<double>((size_t)n * nev) : nullptr;
    void* tws = cv.take<char>(tbytes);
    if (!cv.ok) return SKEW_ERR_WORKSPACE;
    // every scratch word the kernels read is written first in the same call
    // (the failure flag is reset by tridiag_eig), so no clearing is needed
    rc = tridiag_eig(st, n, alpha, nev, lambda, Qi, tws, tbytes, d_status, 5);
    if (rc) return rc;
    if (Q && interleaved_to_colmajor(st, n, nev, Qi, Q, nullptr, ldq, false) != cudaSuccess) return SKEW_ERR_CUDA;
    return cudaGetLastError() == cudaSuccess ? 0 : SKEW_ERR_CUDA;
}
