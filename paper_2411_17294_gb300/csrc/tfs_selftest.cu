// Check of the bounded device wait that every mbarrier wait of the library
// uses (mbar_wait: about 2 s, then it gives up so that a kernel can latch
// TFS_FLAG_TIMEOUT and return instead of hanging).  One thread waits on an
// mbarrier that nothing arrives at; the wait must give up, and the GPU context
// stays usable.  No device memory is allocated: the result words are a
// file-scope __device__ array.
#include <cuda_runtime.h>

#include "../../include/tfs.h"
#include "tfs_device.cuh"

namespace {

__device__ unsigned long long g_wait_check[2];   // flags, elapsed ns

__global__ void wait_bound_kernel() {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        tfs::mbar_init(&bar, 1);
        tfs::fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned long long t0 = tfs::global_ns();
        const bool ok = tfs::mbar_wait(&bar, 0u);     // phase 0 needs one arrival that never comes
        g_wait_check[1] = tfs::global_ns() - t0;
        g_wait_check[0] = ok ? 0ull : (unsigned long long)TFS_FLAG_TIMEOUT;
    }
}

}  // namespace

extern "C" int tfs_check_wait_bound(unsigned* flags, double* seconds, void* stream) {
    if (!flags || !seconds) return TFS_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    wait_bound_kernel<<<1, 32, 0, s>>>();
    unsigned long long out[2] = {0, 0};
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyFromSymbolAsync(out, g_wait_check, sizeof(out), 0, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return TFS_ERR_CUDA;
    *flags = (unsigned)out[0];
    *seconds = (double)out[1] * 1e-9;
    return TFS_OK;
}
