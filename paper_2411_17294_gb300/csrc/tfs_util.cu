// Small helper kernels of libtfs: state initialisation, clearing, checkpoint
// headers, conversions used by the adjoint driver.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "tfs_internal.h"

namespace tfs {

// cuTensorMapEncodeTiled from the driver (through the runtime, so that the
// library links no driver stub); nullptr if the driver does not provide it.
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return (PFN_cuTensorMapEncodeTiled_v12000) nullptr;
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }();
    return fn;
}

namespace {
// Encoded maps are a pure function of their inputs, so the last few are kept:
// a step re-uses the maps of the workspace fields and usually of the caller's
// velocity-gradient buffers.
struct MapKey {
    const void* base;
    long long N;
    int planes, box_h;
    bool dbl;
    bool operator==(const MapKey& o) const {
        return base == o.base && N == o.N && planes == o.planes && box_h == o.box_h && dbl == o.dbl;
    }
};
constexpr int kMapCache = 64;
struct MapCache {
    MapKey key[kMapCache];
    CUtensorMap map[kMapCache];
    bool used[kMapCache] = {};
    int next = 0;
    std::mutex mu;
};
MapCache& map_cache() {
    static MapCache c;
    return c;
}
}  // namespace

bool encode_plane_map(CUtensorMap* map, const void* base, long long N, int planes, int box_h, bool dbl) {
    const size_t es = dbl ? 8 : 4;
    if (!base || (reinterpret_cast<uintptr_t>(base) & 15u) != 0 || N < 1 || planes < 1 || box_h < 1 ||
        box_h > 256 || planes % box_h != 0 || ((size_t)N * es) % 16 != 0)
        return false;
    const MapKey key{base, N, planes, box_h, dbl};
    MapCache& cache = map_cache();
    {
        std::lock_guard<std::mutex> lock(cache.mu);
        for (int i = 0; i < kMapCache; ++i)
            if (cache.used[i] && cache.key[i] == key) {
                *map = cache.map[i];
                return true;
            }
    }
    const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)N, (cuuint64_t)planes};
    const cuuint64_t strides[1] = {(cuuint64_t)N * es};
    const cuuint32_t box[2] = {32u, (cuuint32_t)box_h};
    const cuuint32_t estr[2] = {1u, 1u};
    const CUresult r = enc(map, dbl ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                           const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return false;
    std::lock_guard<std::mutex> lock(cache.mu);
    const int i = cache.next;
    cache.next = (cache.next + 1) % kMapCache;
    cache.key[i] = key;
    cache.map[i] = *map;
    cache.used[i] = true;
    return true;
}

namespace {
struct PlanKey {
    const void* kern;
    int dev, threads;
    size_t stage_bytes, static_bytes;
};
constexpr int kPlanCache = 64;
struct PlanCache {
    PlanKey key[kPlanCache];
    PersistPlan plan[kPlanCache];
    int count = 0;
    // dynamic shared-memory limit set on each (kernel, device): only ever
    // raised, so that it covers every cached plan of that kernel
    const void* attr_kern[kPlanCache];
    int attr_dev[kPlanCache];
    size_t attr_val[kPlanCache];
    int attr_count = 0;
    std::mutex mu;
};
PlanCache& plan_cache() {
    static PlanCache c;
    return c;
}
}  // namespace

cudaError_t persistent_plan(const void* kern, int threads, size_t stage_bytes, size_t static_bytes, int max_stages,
                            PersistPlan* out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    PlanCache& cache = plan_cache();
    std::lock_guard<std::mutex> lock(cache.mu);
    for (int i = 0; i < cache.count; ++i) {
        const PlanKey& k = cache.key[i];
        if (k.kern == kern && k.dev == dev && k.threads == threads && k.stage_bytes == stage_bytes &&
            k.static_bytes == static_bytes) {
            *out = cache.plan[i];
            return cudaSuccess;
        }
    }
    int max_optin = 0, sms = 0;
    e = cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    int ai = 0;
    while (ai < cache.attr_count && !(cache.attr_kern[ai] == kern && cache.attr_dev[ai] == dev)) ++ai;
    if (ai == cache.attr_count) {
        if (ai == kPlanCache) return cudaErrorInvalidConfiguration;
        cache.attr_kern[ai] = kern;
        cache.attr_dev[ai] = dev;
        cache.attr_val[ai] = 0;
        ++cache.attr_count;
    }
    // stage buffers per block: the most tiles staged per SM (buffers x resident
    // blocks) wins -- a second buffer hides the whole load of the next tile,
    // where one buffer exposes the latency of its second half; on a tie the
    // fewer buffers (more resident warps) win
    PersistPlan best{0, 0, sms, 0};
    for (int st = 1; st <= max_stages; ++st) {
        const size_t dyn = (size_t)st * stage_bytes + 128;   // + alignment slack of the stage buffers
        if (dyn + static_bytes > (size_t)max_optin) continue;
        if (dyn > cache.attr_val[ai]) {
            e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
            if (e != cudaSuccess) return e;
            cache.attr_val[ai] = dyn;
        }
        int blocks = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kern, threads, dyn);
        if (e != cudaSuccess) return e;
        if (blocks > 0 && st * blocks > best.stages * best.per_sm) best = PersistPlan{st, blocks, sms, dyn};
    }
    if (best.per_sm < 1) return cudaErrorInvalidConfiguration;
    if (cache.count < kPlanCache) {
        cache.key[cache.count] = PlanKey{kern, dev, threads, stage_bytes, static_bytes};
        cache.plan[cache.count] = best;
        ++cache.count;
    }
    *out = best;
    return cudaSuccess;
}
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
