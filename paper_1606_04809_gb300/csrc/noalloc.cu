// asaga_recompute_abar_noalloc: the float64 recomputation of
// abar = (1/n) sum_i alpha_i a_i for callers that cannot allocate device
// memory.
//
// Who cannot allocate: a process that must keep a fixed device-memory
// footprint reserved up front (a multi-tenant server or a real-time loop,
// where an allocation at run time can fail or stall); code embedded in a
// framework that owns all device memory through its own allocator and
// forbids side allocations; and code on a path where the device-wide
// synchronisation of cudaFree is not acceptable.  Such callers pass every
// input and output in their own device memory, and this function keeps its
// float64 accumulators in a fixed array compiled into the library.
//
// The scratch is a file-scope __device__ array.  In host code its name only
// stands for the symbol, not for a device address, so the first call on each
// device (with that device current) looks the address up once with
// cudaGetSymbolAddress and passes that pointer to the kernels.  The address
// belongs to the device's CUDA context: a cudaDeviceReset destroys that
// context (and the array with it), so the cached address is keyed by the
// context's process-unique id (cuCtxGetId) and looked up again when the
// current context is a different one.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "asaga.h"
#include "asaga_internal.h"
#include "device_common.cuh"

namespace asaga {
namespace {

constexpr int kNoAllocBlocks = 1024;  // blocks of the finishing pass (one partial each)
constexpr int kMaxDevices = 64;

// float64 accumulator per column and one partial maximum per block
__device__ __align__(256) double g_noalloc_acc[ASAGA_NOALLOC_MAX_D];
__device__ __align__(256) double g_noalloc_partial[kNoAllocBlocks];

struct Scratch {
    double *acc = nullptr;
    double *partial = nullptr;
    unsigned long long ctx_id = 0;  // context the addresses belong to (0: none yet)
};
Scratch g_scratch[kMaxDevices];
std::mutex g_scratch_mutex;

// Process-unique id of the calling thread's current CUDA context, 0 when
// there is none yet (or the driver cannot say).  The two driver calls are
// fetched through the runtime, so the library does not link libcuda itself.
unsigned long long current_context_id() {
    using GetCurrent = CUresult (*)(CUcontext *);
    using GetId = CUresult (*)(CUcontext, unsigned long long *);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<GetCurrent>(f);
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<GetId>(f);
    });
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}

// Device addresses of the scratch on the current device: the set-up, once
// per device and context (again after a cudaDeviceReset made a new context).
cudaError_t scratch_for_current_device(Scratch *out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    Scratch &s = g_scratch[dev];
    const unsigned long long id = current_context_id();
    if (!s.acc || !s.partial || id == 0 || id != s.ctx_id) {
        void *acc = nullptr, *partial = nullptr;
        e = cudaGetSymbolAddress(&acc, g_noalloc_acc);
        if (e != cudaSuccess) return e;
        e = cudaGetSymbolAddress(&partial, g_noalloc_partial);
        if (e != cudaSuccess) return e;
        s.acc = static_cast<double *>(acc);
        s.partial = static_cast<double *>(partial);
        s.ctx_id = current_context_id();  // the lookup made the device's context current
    }
    *out = s;
    return cudaSuccess;
}

__global__ void noalloc_zero_kernel(double *acc, int64_t d) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < d; v += (int64_t)gridDim.x * blockDim.x)
        acc[v] = 0.0;
}

__device__ __forceinline__ double block_max(double v) {
    __shared__ double red[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    v = warp_max(v);
    if (lane == 0) red[w] = v;
    __syncthreads();
    double r = 0.0;
    if (w == 0) {
        r = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
        r = warp_max(r);
    }
    return r;  // valid in thread 0
}

// abar_v <- (float)acc_v; partial[b] <- max over the block's columns of |abar_v(in) - acc_v|.
__global__ void noalloc_finish_kernel(const double *acc, float *abar, int64_t d, double *partial) {
    double local = 0.0;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < d; v += (int64_t)gridDim.x * blockDim.x) {
        const double exact = acc[v];
        local = fmax(local, fabs((double)abar[v] - exact));
        abar[v] = (float)exact;
    }
    const double r = block_max(local);
    if (threadIdx.x == 0) partial[blockIdx.x] = r;
}

__global__ void noalloc_max_kernel(const double *partial, int grid, double *out) {
    double v = 0.0;
    for (int j = threadIdx.x; j < grid; j += blockDim.x) v = fmax(v, partial[j]);
    const double r = block_max(v);
    if (threadIdx.x == 0) out[0] = r;
}

asaga_status noalloc_fail(asaga_status s, const std::string &msg) {
    set_thread_error(msg);
    return s;
}

}  // namespace
}  // namespace asaga

using namespace asaga;

extern "C" asaga_status asaga_recompute_abar_noalloc(int64_t n, int64_t d, const int64_t *row_ptr,
                                                     const int32_t *col_idx, const float *values,
                                                     const float *alpha, float *abar, double *drift,
                                                     void *stream) {
    if (n < 1) return noalloc_fail(ASAGA_EINVAL, "n must be >= 1");
    if (d < 1 || d > ASAGA_NOALLOC_MAX_D)
        return noalloc_fail(ASAGA_EINVAL, "d = " + std::to_string(d) + " is outside [1, " +
                                              std::to_string((long long)ASAGA_NOALLOC_MAX_D) +
                                              "], the columns the fixed scratch holds");
    if (!row_ptr || !col_idx || !values || !alpha || !abar)
        return noalloc_fail(ASAGA_EINVAL, "row_ptr, col_idx, values, alpha and abar must not be NULL");
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    Scratch scratch;
    cudaError_t e = scratch_for_current_device(&scratch);
    if (e != cudaSuccess) return noalloc_fail(ASAGA_ECUDA, std::string("scratch address: ") + cudaGetErrorString(e));
    int dev = 0, sms = 1;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return noalloc_fail(ASAGA_ECUDA, std::string("device query: ") + cudaGetErrorString(e));

    EvalParams p{};
    p.n = n;
    p.d = d;
    p.row_ptr = row_ptr;
    p.col_idx = col_idx;
    p.values = values;
    p.alpha = alpha;
    p.stride = 1;
    const int col_grid = (int)std::min<int64_t>(kNoAllocBlocks, std::max<int64_t>(1, (d + 255) / 256));
    const int row_grid = std::min(kMaxPartials, sms * 4);
    noalloc_zero_kernel<<<col_grid, 256, 0, s>>>(scratch.acc, d);
    if ((e = cudaGetLastError()) != cudaSuccess) return noalloc_fail(ASAGA_ECUDA, cudaGetErrorString(e));
    if ((e = launch_scatter_rows(p, kF32, false, 1, row_grid, scratch.acc, s)) != cudaSuccess)
        return noalloc_fail(ASAGA_ECUDA, cudaGetErrorString(e));
    noalloc_finish_kernel<<<col_grid, 256, 0, s>>>(scratch.acc, abar, d, scratch.partial);
    if ((e = cudaGetLastError()) != cudaSuccess) return noalloc_fail(ASAGA_ECUDA, cudaGetErrorString(e));
    if (drift) {
        noalloc_max_kernel<<<1, 256, 0, s>>>(scratch.partial, col_grid, drift);
        if ((e = cudaGetLastError()) != cudaSuccess) return noalloc_fail(ASAGA_ECUDA, cudaGetErrorString(e));
    }
    return ASAGA_OK;
}
