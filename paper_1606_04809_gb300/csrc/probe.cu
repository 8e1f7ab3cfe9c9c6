// asaga_probe_line_rate: the L2 service time of one column's state line under
// the update kernel's own access pattern.
//
// Every update whose row holds column v reads v's 8-byte state {x, abar}
// (the inconsistent read of x^_v in Algorithm 2) and then adds to x_v and
// abar_v with one 2-wide float reduction whose value depends on that read
// (D_v, constant, comes from another array through L1).  All such accesses meet at the one L2 slice that owns the line, which
// serialises them.  A column held by c rows therefore costs an epoch at
// least c times the service time of one (read, reduction) pair, whatever the
// number of warps; on a problem whose most frequent column is in almost every
// row this floor, not HBM bandwidth, is the update kernel's roofline.
//
// The probe runs `warps` warps whose lane 0 repeats the pair `pairs` times on
// one line (the other lanes idle, as the lanes that do not own the column
// do), so the line sees warps x pairs pairs, warps of them in flight at
// once.  Enough warps saturate the line; the elapsed time per pair is then
// its service time.
#include <cuda_runtime.h>

#include <string>

#include "asaga.h"
#include "asaga_internal.h"
#include "device_common.cuh"

namespace asaga {
namespace {

__global__ void line_probe_kernel(float2 *line, int64_t pairs, int warps) {
    const int warp = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
    if (warp >= warps || (threadIdx.x & 31) != 0) return;
    for (int64_t k = 0; k < pairs; ++k) {
        const float2 s = ld_state(line);
        // a value that depends on the read and leaves the line's numbers
        // unchanged in practice (the adds are ~1e-30 of the values read)
        red_add_v2(line, s.x * 1e-30f, s.y * 1e-30f);
    }
}

}  // namespace
}  // namespace asaga

using namespace asaga;

extern "C" asaga_status asaga_probe_line_rate(int warps, int64_t pairs, double *ns_per_pair) {
    if (warps < 1 || warps > (1 << 16) || pairs < 1 || !ns_per_pair) {
        set_thread_error("warps must be in [1, 65536], pairs >= 1 and ns_per_pair not NULL");
        return ASAGA_EINVAL;
    }
    float2 *line = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    cudaStream_t s = nullptr;
    std::string where;
    cudaError_t e = cudaSuccess;
    float ms = 0.f;
    const int block = 256, grid = (warps * 32 + block - 1) / block;
    do {
        if ((e = cudaMalloc(&line, 256)) != cudaSuccess) { where = "alloc"; break; }
        if ((e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) != cudaSuccess) { where = "stream"; break; }
        if ((e = cudaMemsetAsync(line, 0, 256, s)) != cudaSuccess) { where = "memset"; break; }
        if ((e = cudaEventCreate(&a)) != cudaSuccess || (e = cudaEventCreate(&b)) != cudaSuccess) { where = "event"; break; }
        // one short warm-up launch, then the timed one
        line_probe_kernel<<<grid, block, 0, s>>>(line, pairs < 16 ? pairs : 16, warps);
        if ((e = cudaGetLastError()) != cudaSuccess) { where = "launch"; break; }
        if ((e = cudaEventRecord(a, s)) != cudaSuccess) { where = "event record"; break; }
        line_probe_kernel<<<grid, block, 0, s>>>(line, pairs, warps);
        if ((e = cudaGetLastError()) != cudaSuccess) { where = "launch"; break; }
        if ((e = cudaEventRecord(b, s)) != cudaSuccess) { where = "event record"; break; }
        if ((e = cudaEventSynchronize(b)) != cudaSuccess) { where = "synchronize"; break; }
        if ((e = cudaEventElapsedTime(&ms, a, b)) != cudaSuccess) { where = "elapsed"; break; }
    } while (false);
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (s) cudaStreamDestroy(s);
    if (line) cudaFree(line);
    if (e != cudaSuccess) {
        set_thread_error("asaga_probe_line_rate: " + where + ": " + cudaGetErrorString(e));
        return ASAGA_ECUDA;
    }
    *ns_per_pair = (double)ms * 1e6 / ((double)warps * (double)pairs);
    return ASAGA_OK;
}
