// mf_residual_noalloc: r = b - A x for A given element by element, using no
// device allocation at all.
//
// Who needs this: callers that may not call cudaMalloc (or any allocating
// routine) when they evaluate a residual -- code running under a memory
// budget fixed in advance, inside a host framework that owns every device
// allocation through its own pool, or in a real-time loop where an
// allocation's implicit synchronisation is not allowed.  Such callers pass
// their own inputs and output; the only work space is the file-scope array
// below, which a device holds from the moment the library's device code is
// loaded there until the process exits.  Under CUDA's lazy module loading
// (the default) that is the first call of this entry point on the device:
// that set-up call may take device memory once, later calls take none.
//
// Contract (also stated in include/mfsolve.h):
//  * n_dof * nrhs must not exceed MF_NOALLOC_MAX_ENTRIES (1 << 20 doubles,
//    8 MiB); larger calls return MF_ETOOLARGE and launch nothing.
//  * The first call on a device looks up the array's device address with
//    cudaGetSymbolAddress (with that device current) and caches it; make that
//    first call before any stream capture.  The cached address belongs to the
//    CUDA context of that first call: after cudaDeviceReset the process must
//    load the library afresh before calling this again.
//  * All calls share the one array and leave their sums in it; each call
//    clears the part it uses before accumulating.  Calls whose work overlaps
//    on the GPU (other streams, other host threads) race on the array.
//  * Sums are accumulated with FP64 atomics, so the rounding order (not the
//    value beyond rounding) can differ from mf_residual.
//  * nodes_per_elem <= 64 and nrhs <= 65535 (one grid row per right-hand
//    side), else MF_EINVAL before anything is launched.
//  * Every element node id must lie in [0, n_dof).  The kernel checks each id
//    before using it: an id outside that range is neither read through nor
//    written through, a flag in the scratch array is raised, and the call
//    then fills all of d_r with NaN so the caller sees the bad input in the
//    output (the call itself returns before the GPU has run, so it cannot
//    return an error code for it).
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "mfsolve.h"

namespace {

constexpr int kMaxDevices = 64;

// MF_NOALLOC_MAX_ENTRIES sums, then one word for the bad-node-id flag
static __device__ __align__(256) double g_noalloc_scratch[MF_NOALLOC_MAX_ENTRIES + 1];

std::mutex g_setup_mutex;
double* g_scratch_addr[kMaxDevices] = {};

// clears the n sums in use and the bad-id flag (stored at acc[MF_NOALLOC_MAX_ENTRIES])
__global__ void k_noalloc_zero(double* __restrict__ acc, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) acc[i] = 0.0;
    if (i == 0) acc[MF_NOALLOC_MAX_ENTRIES] = 0.0;
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
    const int64_t row = nd[a];
    bool bad = row < 0 || row >= n_dof;
    double s = 0.0;
    for (int b = 0; b < npe; b++) {
        const int64_t c = nd[b];
        if (c < 0 || c >= n_dof) {
            bad = true;
            continue;
        }
        s = fma(K[b * npe], xr[c], s);
    }
    if (bad) {
        acc[MF_NOALLOC_MAX_ENTRIES] = 1.0;  // benign race: every writer stores the same value
        return;
    }
    atomicAdd(acc + (int64_t)r * n_dof + row, s);
}

__global__ void k_noalloc_finish(const double* __restrict__ b, const double* __restrict__ acc, double* __restrict__ r,
                                 int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) r[i] = acc[MF_NOALLOC_MAX_ENTRIES] != 0.0 ? __longlong_as_double(0x7ff8000000000000ll) : b[i] - acc[i];
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
    if (n_dof < 1 || n_elem < 1 || nodes_per_elem < 1 || nodes_per_elem > 64 || nrhs < 1 || nrhs > 65535)
        return MF_EINVAL;
    if (!d_elem_nodes || !d_values || !d_x || !d_b || !d_r) return MF_EINVAL;
    if (n_dof > (int64_t)MF_NOALLOC_MAX_ENTRIES / nrhs) return MF_ETOOLARGE;
    const int64_t nE = n_elem * nodes_per_elem;
    if ((nE + 255) / 256 > 0x7fffffffll) return MF_ETOOLARGE;  // grid x limit of the element kernel
    double* acc = nullptr;
    int rc = scratch_for_current_device(&acc);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = n_dof * nrhs;
    // each launch is checked before the next is issued, so d_r is never written after a failed step
    k_noalloc_zero<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(acc, n);
    if (cudaGetLastError() != cudaSuccess) return MF_ECUDA;
    dim3 g((unsigned)((nE + 255) / 256), nrhs);
    k_noalloc_apply<<<g, 256, 0, s>>>(d_values, d_elem_nodes, d_x, acc, n_elem, nodes_per_elem, n_dof);
    if (cudaGetLastError() != cudaSuccess) return MF_ECUDA;
    k_noalloc_finish<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(d_b, acc, d_r, n);
    if (cudaGetLastError() != cudaSuccess) return MF_ECUDA;
    return MF_OK;
}
