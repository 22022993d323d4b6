// Small helper kernels of libtfs: state initialisation, clearing, checkpoint
// headers, conversions used by the adjoint driver.
#include <cuda_runtime.h>
#include <stdint.h>

#include "tfs_internal.h"

namespace tfs {
namespace {

template <typename T>
__global__ void fill_levels_kernel(T* a, T* b, T* c, const T* src, long long count) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x) {
        const T v = src ? src[i] : (T)0;
        a[i] = v;
        b[i] = v;
        if (c) c[i] = v;
    }
}

__global__ void zero_kernel(uint4* p, long long n16, unsigned char* tail, int ntail) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n16;
         i += (long long)gridDim.x * blockDim.x)
        p[i] = make_uint4(0, 0, 0, 0);
    if (blockIdx.x == 0 && (int)threadIdx.x < ntail) tail[threadIdx.x] = 0;
}

struct Words { uint64_t w[16]; };

__global__ void header_kernel(uint64_t* dst, Words words, int count) {
    if ((int)threadIdx.x < count) dst[threadIdx.x] = words.w[threadIdx.x];
}

template <typename T>
__global__ void to_double_kernel(const T* src, double* dst, long long count) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x)
        dst[i] = (double)src[i];
}

__global__ void add_initial_kernel(double* g, const double* s1, const double* s0, long long count) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x)
        g[i] += s1[i] + s0[i];
}

unsigned grid_for(long long count) {
    long long b = (count + 255) / 256;
    if (b < 1) b = 1;
    if (b > 152 * 64) b = 152 * 64;
    return (unsigned)b;
}

}  // namespace

cudaError_t launch_fill_levels(void* sig_n, void* sig_nm1, void* sigma0_copy, const void* sigma0,
                               long long count, bool is_double, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    if (is_double)
        fill_levels_kernel<double><<<grid_for(count), 256, 0, s>>>((double*)sig_n, (double*)sig_nm1,
                                                                  (double*)sigma0_copy, (const double*)sigma0, count);
    else
        fill_levels_kernel<float><<<grid_for(count), 256, 0, s>>>((float*)sig_n, (float*)sig_nm1,
                                                                 (float*)sigma0_copy, (const float*)sigma0, count);
    return cudaGetLastError();
}

cudaError_t launch_zero(void* p, size_t bytes, cudaStream_t s) {
    if (bytes == 0) return cudaSuccess;
    const long long n16 = (long long)(bytes / 16);
    const int ntail = (int)(bytes % 16);
    zero_kernel<<<grid_for(n16 > 0 ? n16 : 1), 256, 0, s>>>((uint4*)p, n16, (unsigned char*)p + n16 * 16, ntail);
    return cudaGetLastError();
}

cudaError_t launch_write_header(uint64_t* dst, const uint64_t* words, int count, cudaStream_t s) {
    if (count > 16) return cudaErrorInvalidValue;
    Words w{};
    for (int i = 0; i < count; ++i) w.w[i] = words[i];
    header_kernel<<<1, 32, 0, s>>>(dst, w, count);
    return cudaGetLastError();
}

cudaError_t launch_to_double(const void* src, double* dst, long long count, bool is_double, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    if (is_double)
        to_double_kernel<double><<<grid_for(count), 256, 0, s>>>((const double*)src, dst, count);
    else
        to_double_kernel<float><<<grid_for(count), 256, 0, s>>>((const float*)src, dst, count);
    return cudaGetLastError();
}

cudaError_t launch_add_initial(double* g_sigma0, const double* s1, const double* s0, long long count,
                               cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    add_initial_kernel<<<grid_for(count), 256, 0, s>>>(g_sigma0, s1, s0, count);
    return cudaGetLastError();
}

}  // namespace tfs
