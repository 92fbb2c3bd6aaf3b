// rac_noalloc.cu - random assembly without any device allocation.
//
// rac_assembly() obtains its scratch (the sort keys and indices) from
// cudaMallocAsync on every call.  Some callers cannot allocate: code whose
// device memory is entirely owned by its own allocator (a framework's caching
// allocator that must see every byte), or latency-critical loops where an
// allocation could synchronise with other work on the device.  For them,
// rac_assembly_noalloc() runs the same assembly with its scratch in one
// file-scope device array of fixed size, which every GPU that loads this
// library holds until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "rac_device.cuh"
#include "rac_internal.h"

namespace rac {

// Scratch for up to RAC_ASSEMBLY_NOALLOC_MAX (coordinate, sweep) pairs: one
// 64-bit key and one 32-bit index each (12 bytes per pair, 3 MiB in total).
static __device__ __align__(256) unsigned char g_assembly_scratch[(size_t)RAC_ASSEMBLY_NOALLOC_MAX * 12];

// Same work as k_assembly, with the scratch pointer passed in.  Every scratch
// entry this kernel reads was written earlier in the same launch, so nothing
// in the array has to start at zero.
__global__ void __launch_bounds__(1024) k_assembly_noalloc(int n, int p, uint64_t seed,
                                                           int64_t sweep0, int *perm, int *blk,
                                                           unsigned char *scratch, int L) {
    extern __shared__ unsigned sm_u[];
    const int slot = blockIdx.x;
    uint64_t *tkey = (uint64_t *)scratch;
    int *tidx = (int *)(scratch + (size_t)RAC_ASSEMBLY_NOALLOC_MAX * 8);
    assemble_one(n, p, seed, (uint64_t)(sweep0 + slot), perm + (size_t)slot * n,
                 blk ? blk + (size_t)slot * n : nullptr, tkey + (size_t)slot * n,
                 tidx + (size_t)slot * n, L, sm_u);
}

// Device address of the scratch array, looked up once per device with that
// device current (the host-side symbol is only a stand-in, not an address).
// The address belongs to the device's primary context: a cudaDeviceReset()
// of the device invalidates it (the header tells callers not to use the
// library on a device after a reset).
constexpr int kMaxDevices = 64;
static std::mutex g_mu;
static void *g_addr[kMaxDevices] = {nullptr};

static cudaError_t scratch_address(int dev, void **out) {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_assembly_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = ptr;
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

}  // namespace rac

using namespace rac;

extern "C" rac_status rac_assembly_noalloc(int64_t n, int32_t num_blocks, uint64_t seed,
                                           int64_t sweep0, int32_t nsweeps, int32_t *perm_out,
                                           int32_t *blk_out, void *stream) {
    if (n <= 0 || num_blocks < 1 || num_blocks > n || nsweeps <= 0 || !perm_out)
        return RAC_ERR_ARG;
    if (n * (int64_t)nsweeps > RAC_ASSEMBLY_NOALLOC_MAX) return RAC_ERR_ARG;
    // Every CUDA call below is checked through its own return code, so an
    // error the caller left pending is neither cleared nor taken for ours.
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return RAC_ERR_CUDA;
    void *scratch = nullptr;
    if (scratch_address(dev, &scratch) != cudaSuccess) return RAC_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    const int L = assembly_log2_buckets((int)n);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)nsweeps);
    cfg.blockDim = dim3(1024);
    cfg.dynamicSmemBytes = (size_t)(3 * (1 << L) + 32) * sizeof(unsigned);
    cfg.stream = st;
    if (cudaLaunchKernelEx(&cfg, k_assembly_noalloc, (int)n, (int)num_blocks, seed, sweep0,
                           (int *)perm_out, (int *)blk_out, (unsigned char *)scratch, L) !=
        cudaSuccess)
        return RAC_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return RAC_ERR_CUDA;
    return RAC_OK;
}
