// lbpf_mass_noalloc: the FP64 field sums of lbpf_mass for callers that cannot
// allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is off limits, such as a host
// callback that must not trigger allocation, a real-time monitor that may not
// block on the allocator, or an embedding runtime that owns every byte of device
// memory and forbids hidden allocations.  Those callers bring their own input
// and output buffers; the only scratch this path uses is the file-scope device
// array below, which exists from the moment the library is loaded on a GPU
// until the process exits.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>
#include <string>

#include "lbpf.h"
#include "step_kernels.cuh"

// Defined in lbpf.cu: the calling thread's message behind lbpf_last_error(NULL).
void lbpf_internal_set_thread_error(const std::string& msg);

namespace {

// 256 threads x 64 elements: one block owns one contiguous chunk of the input.
constexpr int kChunkPerThread = 64;
constexpr long long kChunk = (long long)lbpf::kMassThreads * kChunkPerThread;
constexpr int kMaxBlocks = (int)(LBPF_NOALLOC_MAX_ELEMENTS / kChunk);
static_assert(LBPF_NOALLOC_MAX_ELEMENTS % kChunk == 0, "the element limit is a whole number of chunks");

// Three partial sums per block (sum c, sum phi, count of bad values).  Every
// block overwrites its own three slots before the final pass reads them, so
// nothing in here has to start at zero.
static __device__ __align__(256) double g_noalloc_partials[3 * kMaxBlocks];

// Device addresses of g_noalloc_partials already looked up, keyed by the CUDA
// context they belong to (its process-unique id), so that a device reset or a
// caller's own context never reuses an address from another context.
constexpr int kMaxContexts = 64;
struct CachedAddress {
    unsigned long long ctx_id;
    double* ptr;
};
std::mutex g_setup_mutex;
CachedAddress g_cache[kMaxContexts];
int g_cache_used = 0;

lbpf_status noalloc_fail(lbpf_status st, const std::string& m) {
    lbpf_internal_set_thread_error(m);   // read back with lbpf_last_error(NULL)
    return st;
}

// Each block sums its own chunk [b * kChunk, (b + 1) * kChunk) of both fields.
template <typename R>
__global__ void __launch_bounds__(lbpf::kMassThreads)
k_mass_partial_chunked(const R* __restrict__ c, const R* __restrict__ phi, long long n, double* __restrict__ partials) {
    double sc = 0.0, sp = 0.0, bad = 0.0;
    const long long begin = blockIdx.x * kChunk;
    const long long end = begin + kChunk < n ? begin + kChunk : n;
    for (long long i = begin + threadIdx.x; i < end; i += lbpf::kMassThreads) {
        const double cv = (double)c[i], pv = (double)phi[i];
        sc += cv;
        sp += pv;
        if (!(pv >= -0.5 && pv <= 1.5) || !(cv == cv && cv - cv == 0.0)) bad += 1.0;
    }
    lbpf::block_sum3<R>(sc, sp, bad);
    if (threadIdx.x == 0) {
        partials[3 * blockIdx.x + 0] = sc;
        partials[3 * blockIdx.x + 1] = sp;
        partials[3 * blockIdx.x + 2] = bad;
    }
}

// The id of the calling thread's current CUDA context (0 when there is none),
// through driver entry points fetched once from the runtime.
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

lbpf_status current_context_id(unsigned long long* id) {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    if (!get_current || !get_id) {
        void* f1 = nullptr;
        void* f2 = nullptr;
        cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = q1;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1);
        if (e == cudaSuccess) e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2);
        if (e != cudaSuccess || q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
            return noalloc_fail(LBPF_ECUDA, "driver entry points cuCtxGetCurrent / cuCtxGetId unavailable");
        get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
        get_id = reinterpret_cast<CtxGetIdFn>(f2);
    }
    CUcontext ctx = nullptr;
    if (get_current(&ctx) != CUDA_SUCCESS) return noalloc_fail(LBPF_ECUDA, "cuCtxGetCurrent failed");
    *id = 0;
    if (ctx && get_id(ctx, id) != CUDA_SUCCESS) return noalloc_fail(LBPF_ECUDA, "cuCtxGetId failed");
    return LBPF_OK;
}

// Device address of g_noalloc_partials in the current context.  In host code
// the symbol's name is only a host-side stand-in, so the address is looked up
// once per context (cudaGetSymbolAddress, with that context current, which also
// makes the device's primary context current if no context was) and cached
// under the context's id.
lbpf_status partials_for_current_context(double** out) {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    unsigned long long id = 0;
    lbpf_status st = current_context_id(&id);
    if (st != LBPF_OK) return st;
    for (int i = 0; id != 0 && i < g_cache_used; ++i)
        if (g_cache[i].ctx_id == id) {
            *out = g_cache[i].ptr;
            return LBPF_OK;
        }
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess || !p)
        return noalloc_fail(LBPF_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    if (id == 0 && (st = current_context_id(&id)) != LBPF_OK) return st;   // the lookup made one current
    if (id != 0) {
        // a full table overwrites the slot the id selects; a context whose
        // entry was overwritten simply looks its address up again
        const int slot = g_cache_used < kMaxContexts ? g_cache_used++ : (int)(id % kMaxContexts);
        g_cache[slot] = CachedAddress{id, static_cast<double*>(p)};
    }
    *out = static_cast<double*>(p);
    return LBPF_OK;
}

}  // namespace

extern "C" lbpf_status lbpf_mass_noalloc(const void* c, const void* phi, int64_t n, int32_t precision,
                                         double* out_device, void* cuda_stream) {
    if (!c || !phi || !out_device) return noalloc_fail(LBPF_EINVAL, "NULL input or output pointer");
    if (precision != LBPF_FP64 && precision != LBPF_FP32)
        return noalloc_fail(LBPF_EINVAL, "precision must be LBPF_FP64 or LBPF_FP32");
    if (n < 0) return noalloc_fail(LBPF_EINVAL, "n < 0");
    const long long max_n = (long long)kMaxBlocks * kChunk;
    if (n > max_n) {
        char buf[160];
        snprintf(buf, sizeof(buf), "n = %lld exceeds the no-alloc maximum of %lld elements (%d blocks x %lld)",
                 (long long)n, max_n, kMaxBlocks, kChunk);
        return noalloc_fail(LBPF_EINVAL, buf);
    }
    double* partials = nullptr;
    lbpf_status st = partials_for_current_context(&partials);
    if (st != LBPF_OK) return st;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int blocks = (int)((n + kChunk - 1) / kChunk);
    if (blocks > 0) {
        if (precision == LBPF_FP64)
            k_mass_partial_chunked<double><<<blocks, lbpf::kMassThreads, 0, s>>>(
                (const double*)c, (const double*)phi, n, partials);
        else
            k_mass_partial_chunked<float><<<blocks, lbpf::kMassThreads, 0, s>>>(
                (const float*)c, (const float*)phi, n, partials);
    }
    lbpf::k_mass_final<<<1, lbpf::kMassThreads, 0, s>>>(partials, blocks, out_device);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return noalloc_fail(LBPF_ECUDA, std::string("mass kernels: ") + cudaGetErrorString(e));
    return LBPF_OK;
}
