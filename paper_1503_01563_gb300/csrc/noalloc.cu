// tvcut_iterate_noalloc: product-space iterations on caller-owned device
// buffers, for callers that cannot let the library allocate device memory --
// for example code that runs inside a framework whose allocator owns all of
// the GPU's memory, or a latency-critical loop where a cudaMalloc (which may
// synchronise the device) is not acceptable.  The only scratch the iteration
// needs, the per-vertex running sum of one iteration's sweeps, lives in the
// file-scope device array below instead of a cudaMalloc'd buffer.
//
// The array is part of the library image: every GPU on which the library is
// loaded holds its 8 MiB until the process exits.  All calls share it, so
// calls that overlap on the GPU (different streams, or different host
// threads on the same device) race on it.  Each iteration writes the whole
// running sum before reading it, so nothing has to be cleared between calls.
#include <string.h>

#include <mutex>
#include <string>

#include "tvcut_internal.cuh"

namespace tvcut {
void set_thread_error(const std::string& msg);
}

using namespace tvcut;

namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)8 << 20;   // 2^21 FP32 or 2^20 FP64 values
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device (with that device current) and cached.
tvcut_status scratch_address(void** out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        set_thread_error(std::string("tvcut_iterate_noalloc: cudaGetDevice: ") + cudaGetErrorString(e));
        return TVCUT_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        set_thread_error("tvcut_iterate_noalloc: device ordinal beyond 63");
        return TVCUT_ERR_INVALID;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            set_thread_error(std::string("tvcut_iterate_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            return TVCUT_ERR_CUDA;
        }
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return TVCUT_OK;
}

template <typename T>
tvcut_status run(int ndim, const int64_t* dims, int algo, const void* w, const void* const* a, void* state,
                 void* x, int64_t iters, cudaStream_t stream, void* scratch)
{
    int64_t n = 1;
    for (int k = 0; k < ndim; ++k) n *= dims[k];
    const bool aar = algo == TVCUT_AAR;
    const int first = aar ? MODE_AAR_FIRST : MODE_AP_FIRST;
    const int mid = aar ? MODE_AAR_MID : MODE_AP_MID;
    const int last = aar ? MODE_AAR_LAST : MODE_AP_LAST;
    for (int64_t it = 0; it < iters; ++it) {
        const int check = (x != nullptr && it == iters - 1) ? 1 : 0;
        for (int k = 0; k < ndim; ++k) {
            SweepArgs<T> A;
            memset(&A, 0, sizeof(A));
            A.g = chain_geom(ndim, dims, k);
            A.v = (const T*)state + k * n;
            A.a = (const T*)a[k];
            A.out = (T*)state + k * n;
            A.P = (T*)scratch;
            A.w = (const T*)w;
            for (int j = 0; j < ndim; ++j) A.Z[j] = (T*)state + j * n;
            A.x = (T*)x;
            A.r = ndim;
            A.check = check;
            A.mapping = -1;
            const int mode = k == 0 ? first : (k == ndim - 1 ? last : mid);
            cudaError_t e = launch_sweep<T>(mode, A, stream);
            if (e != cudaSuccess) {
                set_thread_error(std::string("tvcut_iterate_noalloc: launch: ") + cudaGetErrorString(e));
                return TVCUT_ERR_CUDA;
            }
        }
    }
    return TVCUT_OK;
}

}  // namespace

extern "C" tvcut_status tvcut_iterate_noalloc(int ndim, const int64_t* dims, int algo, int dtype,
                                              const void* w, const void* const* a, void* state, void* x,
                                              int64_t iters, void* cuda_stream)
{
    if (ndim != 2 && ndim != 3) {
        set_thread_error("tvcut_iterate_noalloc: ndim must be 2 or 3");
        return TVCUT_ERR_INVALID;
    }
    if (!dims || !w || !a || !state) {
        set_thread_error("tvcut_iterate_noalloc: NULL pointer argument");
        return TVCUT_ERR_INVALID;
    }
    if (algo != TVCUT_AAR && algo != TVCUT_AP) {
        set_thread_error("tvcut_iterate_noalloc: algo must be TVCUT_AAR or TVCUT_AP");
        return TVCUT_ERR_INVALID;
    }
    if (dtype != TVCUT_F32 && dtype != TVCUT_F64) {
        set_thread_error("tvcut_iterate_noalloc: dtype must be TVCUT_F32 or TVCUT_F64");
        return TVCUT_ERR_INVALID;
    }
    if (iters < 0) {
        set_thread_error("tvcut_iterate_noalloc: iters must be >= 0");
        return TVCUT_ERR_INVALID;
    }
    int64_t n = 1;
    for (int k = 0; k < ndim; ++k) {
        if (dims[k] < 1 || dims[k] > ((int64_t)1 << 30)) {
            set_thread_error("tvcut_iterate_noalloc: every dims[k] must be in [1, 2^30]");
            return TVCUT_ERR_INVALID;
        }
        if (dims[k] > 1 && !a[k]) {
            set_thread_error("tvcut_iterate_noalloc: NULL edge-weight pointer");
            return TVCUT_ERR_INVALID;
        }
        n *= dims[k];
        if (n > ((int64_t)1 << 40)) break;
    }
    const size_t esize = dtype == TVCUT_F64 ? 8 : 4;
    if (n > (int64_t)(kNoAllocScratchBytes / esize)) {
        set_thread_error("tvcut_iterate_noalloc: grid has " + std::to_string((long long)n) +
                         " vertices; the no-allocation path holds at most " +
                         std::to_string((long long)(kNoAllocScratchBytes / esize)) +
                         (dtype == TVCUT_F64 ? " (FP64)" : " (FP32)"));
        return TVCUT_ERR_INVALID;
    }
    void* scratch = nullptr;
    tvcut_status st = scratch_address(&scratch);
    if (st != TVCUT_OK) return st;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (dtype == TVCUT_F64) return run<double>(ndim, dims, algo, w, a, state, x, iters, s, scratch);
    return run<float>(ndim, dims, algo, w, a, state, x, iters, s, scratch);
}
