// mf_residual_noalloc: r = b - A x for A given element by element, using no
// device allocation at all.
//
// Who needs this: callers that may not call cudaMalloc (or any allocating
// routine) when they evaluate a residual -- code running under a memory
// budget fixed in advance, inside a host framework that owns every device
// allocation through its own pool, or in a real-time loop where an
// allocation's implicit synchronisation is not allowed.  Such callers pass
// their own inputs and output; the only work space is the file-scope array
// below, which the library's module holds on every device that loads it
// until the process exits.
//
// Contract (also stated in include/mfsolve.h):
//  * n_dof * nrhs must not exceed MF_NOALLOC_MAX_ENTRIES (1 << 20 doubles,
//    8 MiB); larger calls return MF_ETOOLARGE and launch nothing.
//  * The first call on a device looks up the array's device address with
//    cudaGetSymbolAddress (with that device current) and caches it; make that
//    first call before any stream capture.
//  * All calls share the one array and leave their sums in it; each call
//    clears the part it uses before accumulating.  Calls whose work overlaps
//    on the GPU (other streams, other host threads) race on the array.
//  * Sums are accumulated with FP64 atomics, so the rounding order (not the
//    value beyond rounding) can differ from mf_residual.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "mfsolve.h"

namespace {

constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_scratch[MF_NOALLOC_MAX_ENTRIES];

std::mutex g_setup_mutex;
double* g_scratch_addr[kMaxDevices] = {};

__global__ void k_noalloc_zero(double* __restrict__ acc, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) acc[i] = 0.0;
}

// one thread per (element, local row, rhs): acc[node(e,a)] += sum_b K_e[a,b] x[node(e,b)]
__global__ void k_noalloc_apply(const double* __restrict__ values, const int64_t* __restrict__ en,
                                const double* __restrict__ x, double* __restrict__ acc, int64_t n_elem, int npe,
                                int64_t n_dof) {
    const int64_t nE = n_elem * npe;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (idx >= nE) return;
    const int64_t e = idx / npe;
    const int a = (int)(idx - e * npe);
    const double* K = values + e * npe * npe + a;
    const int64_t* nd = en + e * npe;
    const double* xr = x + (int64_t)r * n_dof;
    double s = 0.0;
    for (int b = 0; b < npe; b++) s = fma(K[b * npe], xr[nd[b]], s);
    atomicAdd(acc + (int64_t)r * n_dof + nd[a], s);
}

__global__ void k_noalloc_finish(const double* __restrict__ b, const double* __restrict__ acc, double* __restrict__ r,
                                 int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) r[i] = b[i] - acc[i];
}

// Device address of the scratch array for the current device (looked up once).
int scratch_for_current_device(double** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return MF_ECUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) return MF_ENOTSUP;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            (void)cudaGetLastError();
            return MF_ECUDA;
        }
        g_scratch_addr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_addr[dev];
    return MF_OK;
}

}  // namespace

extern "C" int mf_residual_noalloc(int64_t n_dof, int64_t n_elem, int nodes_per_elem, const int64_t* d_elem_nodes,
                                   const double* d_values, const double* d_x, const double* d_b, double* d_r, int nrhs,
                                   mf_stream_t stream) {
    if (n_dof < 1 || n_elem < 1 || nodes_per_elem < 1 || nodes_per_elem > 64 || nrhs < 1) return MF_EINVAL;
    if (!d_elem_nodes || !d_values || !d_x || !d_b || !d_r) return MF_EINVAL;
    if (n_dof > (int64_t)MF_NOALLOC_MAX_ENTRIES / nrhs) return MF_ETOOLARGE;
    double* acc = nullptr;
    int rc = scratch_for_current_device(&acc);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = n_dof * nrhs;
    const int64_t nE = n_elem * nodes_per_elem;
    k_noalloc_zero<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(acc, n);
    dim3 g((unsigned)((nE + 255) / 256), nrhs);
    k_noalloc_apply<<<g, 256, 0, s>>>(d_values, d_elem_nodes, d_x, acc, n_elem, nodes_per_elem, n_dof);
    k_noalloc_finish<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(d_b, acc, d_r, n);
    if (cudaGetLastError() != cudaSuccess) return MF_ECUDA;
    return MF_OK;
}
