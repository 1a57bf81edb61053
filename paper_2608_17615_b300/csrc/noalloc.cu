// Allocation-free pair sum (ls_pairsum_noalloc).
//
// Some callers cannot call cudaMalloc at all: plug-ins of host applications
// whose device memory is owned by an outside allocator (or a fixed pool
// budgeted up front), and real-time loops that must not enter the driver's
// allocator, whose latency is unbounded.  The regular
// entry points allocate their scratch (the chunked partial sums of the pair
// sum) inside ls_operator_create; this one keeps that scratch in a file-scope
// device array instead, so the call itself allocates nothing.  The paper has
// no counterpart: it is a deployment convenience around the same kernel.
//
// The array is a static __device__ symbol of LS_NOALLOC_SCRATCH double2 (16 MiB);
// every GPU that loads the library holds it until the process exits.  Host
// code cannot use the symbol's name as a device address, so the address is
// looked up with cudaGetSymbolAddress once per device (on the first call made
// with that device current) and cached.  Make that first call before any
// stream capture.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <mutex>
#include <string>

#include "../../include/lsgpu.h"

// Defined in lsgpu.cu: the pair-sum kernel with the direct H0 routine, the
// chunk reduction, and the thread-local error message of ls_last_error().
__global__ void k_pairsum(const double2* xy, const double* w, const double2* m, const double2* f, int n,
                          int src_per_chunk, double k, double inv_k, double2* partial);
__global__ void k_apply_epi(int n, int nchunk, const double2* partial, const int64_t* rowptr, const int* cols,
                            const double2* vals, const double2* m, const double2* x, double k2, double2* y, int mode);
ls_status lsgpu_set_error(ls_status s, const char* msg);
#define ls_internal_fail lsgpu_set_error

#define LS_NOALLOC_SCRATCH (1 << 20)
#define LS_NOALLOC_MAX_DEVICES 64

static __device__ __align__(256) double2 g_noalloc_scratch[LS_NOALLOC_SCRATCH];

static std::mutex g_noalloc_mu;
static double2* g_noalloc_ptr[LS_NOALLOC_MAX_DEVICES] = {};

extern "C" ls_status ls_pairsum_noalloc(int32_t n, const double* xy_dev, const double* w_dev, const void* f_dev,
                                        double k, void* y_dev, void* stream) {
    if (n < 2 || !xy_dev || !w_dev || !f_dev || !y_dev) return ls_internal_fail(LS_EINVAL, "ls_pairsum_noalloc: null pointer or n < 2");
    if (!(k > 0)) return ls_internal_fail(LS_EINVAL, "ls_pairsum_noalloc: k must be positive");
    if (n > LS_NOALLOC_SCRATCH)
        return ls_internal_fail(LS_EINVAL, "ls_pairsum_noalloc: n exceeds the static scratch capacity of 1048576 nodes");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= LS_NOALLOC_MAX_DEVICES)
        return ls_internal_fail(LS_ECUDA, "ls_pairsum_noalloc: no usable current device");
    double2* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void* p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess) return ls_internal_fail(LS_ECUDA, cudaGetErrorString(e));
            g_noalloc_ptr[dev] = static_cast<double2*>(p);
        }
        scratch = g_noalloc_ptr[dev];
    }
    // Source chunks: about 8 blocks of 128 targets per SM, limited by the scratch size.
    int nsm = 148;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int tblocks = (n + 127) / 128;
    int nchunk = (nsm * 8 + tblocks - 1) / tblocks;
    nchunk = std::max(1, std::min(nchunk, std::min(64, LS_NOALLOC_SCRATCH / n)));
    int spc = (n + nchunk - 1) / nchunk;
    spc = ((spc + 255) / 256) * 256;
    nchunk = (n + spc - 1) / spc;
    // Every (chunk, target) partial is written before it is read, so nothing needs clearing.
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    dim3 grid(tblocks, nchunk);
    k_pairsum<<<grid, 128, 0, st>>>(reinterpret_cast<const double2*>(xy_dev), w_dev, nullptr,
                                    static_cast<const double2*>(f_dev), n, spc, k, 1.0 / k, scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return ls_internal_fail(LS_ECUDA, cudaGetErrorString(e));
    const int threads = 256;
    const int blocks = (int)(((int64_t)n * 32 + threads - 1) / threads);
    k_apply_epi<<<blocks, threads, 0, st>>>(n, nchunk, scratch, nullptr, nullptr, nullptr, nullptr, nullptr, 0.0,
                                            static_cast<double2*>(y_dev), 1);
    e = cudaGetLastError();
    if (e != cudaSuccess) return ls_internal_fail(LS_ECUDA, cudaGetErrorString(e));
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return ls_internal_fail(LS_ECUDA, cudaGetErrorString(e));
    return LS_OK;
}
