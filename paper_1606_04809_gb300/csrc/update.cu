// The asynchronous Sparse SAGA update kernel (Algorithm 2 of arXiv:1606.04809
// with the projected l2 term of Sec. 4.2).
//
// Each warp is one ASAGA "core".  Update t of a launch samples its row
// i = sample_row(seed, t) before reading anything (Algorithm 2 samples, then
// reads), reads x^, abar and D on S_i and the memory alpha^_i
// inconsistently (other warps keep adding to them), forms
//     delta = phi'_i(a_i.x^) - alpha^_i,
// and adds, atomically at L2,
//     x_v    += -gamma (delta a_iv + D_v (abar_v + lambda x^_v)),
//     abar_v += delta a_iv / n              for v in S_i,
//     alpha_i += delta                      (Algorithm 2 increments alpha_i by delta-alpha).
// Because alpha_i and abar receive exactly matching increments,
// abar = (1/n) sum_i alpha_i a_i holds in exact arithmetic under any
// interleaving of warps.
//
// Latency: the CSR slice of a row does not depend on the solver state, so a
// warp requests the column indices and values of a row two rows before it
// processes it (and the row_ptr entries three rows before); the window
// between reading x^ and writing x, which sets the overlap tau, is then one
// L2 gather, a warp reduction and the reductions back to L2.
//
// Layout: A in CSR (int64 row_ptr, int32 col_idx, values in fp32/bf16/fp16)
// or dense row-major; per-column state float4 {x, abar, D, 0}, so one
// 16-byte L2 read serves x^_v, abar_v and D_v and one 8-byte vector
// reduction updates x_v and abar_v.  Up to 32 * kSlots entries of a row are
// held in registers (lane l owns entries l, l+32, ...); longer rows read
// the remainder again from memory.
#include "asaga_internal.h"
#include "device_common.cuh"

namespace asaga {

constexpr int kSlots = 4;

// The part of a row that does not depend on the solver state.
struct RowData {
    int64_t start;
    int len;
    float label;
    int c[kSlots];
    float a[kSlots];
};

__device__ __forceinline__ void red_add_f32(float *p, float v) {
    asm volatile("red.relaxed.gpu.global.add.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
}

template <bool kDense>
__device__ __forceinline__ void load_meta(const UpdateParams &P, int64_t i, RowData &r) {
    if (kDense) {
        r.start = i * P.d;
        r.len = (int)P.d;
    } else {
        const int64_t s = __ldg(P.row_ptr + i);
        r.start = s;
        r.len = (int)(__ldg(P.row_ptr + i + 1) - s);
    }
    r.label = __ldg(P.labels + i);
}

template <typename T, bool kDense>
__device__ __forceinline__ void load_slots(const UpdateParams &P, const T *__restrict__ vals, RowData &r,
                                           int lane) {
#pragma unroll
    for (int s = 0; s < kSlots; ++s) {
        const int k = lane + 32 * s;
        r.c[s] = 0;
        r.a[s] = 0.f;
        if (k < r.len) {
            r.c[s] = kDense ? k : ld_stream(P.col_idx + r.start + k);
            r.a[s] = to_f32(ld_stream(vals + r.start + k));
        }
    }
}

// Row of update t of this launch, or -1 past the end (or on a bad index).
__device__ __forceinline__ int64_t row_of(const UpdateParams &P, int64_t t, bool &bad) {
    if (t >= P.count) return -1;
    if (P.idx) {
        const int64_t i = __ldg(P.idx + t);
        if (i < 0 || i >= P.n) {
            bad = true;
            return -1;
        }
        return i;
    }
    return sample_row(P.seed, P.t_begin + (uint64_t)t, P.n);
}

template <typename T, bool kDense>
__device__ __forceinline__ void process_row(const UpdateParams &P, const T *__restrict__ vals, int64_t i,
                                            const RowData &r, int lane) {
    const float4 *__restrict__ state = P.state;
    const int64_t stride = P.stride;
    float4 s[kSlots];
#pragma unroll
    for (int q = 0; q < kSlots; ++q) {
        s[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (lane + 32 * q < r.len) s[q] = ld_state(state + r.c[q] * stride);
    }
    const float alpha_hat = __ldcg(P.alpha + i);
    float z = 0.f;
#pragma unroll
    for (int q = 0; q < kSlots; ++q) z = fmaf(r.a[q], s[q].x, z);
    for (int k = lane + 32 * kSlots; k < r.len; k += 32) {  // rest of a long row
        const int cc = kDense ? k : ld_stream(P.col_idx + r.start + k);
        z = fmaf(to_f32(ld_stream(vals + r.start + k)), ld_state(state + cc * stride).x, z);
    }
    z = warp_sum(z);
    const float delta = phi_prime_f32(P.loss, z, r.label) - alpha_hat;  // same value in every lane

    const float gamma = P.gamma, lambda = P.lambda, inv_n = P.inv_n;
#pragma unroll
    for (int q = 0; q < kSlots; ++q) {
        if (lane + 32 * q < r.len) {
            const float dx = -gamma * fmaf(delta, r.a[q], s[q].z * fmaf(lambda, s[q].x, s[q].y));
            red_add_v2(P.state + r.c[q] * stride, dx, delta * r.a[q] * inv_n);
        }
    }
    for (int k = lane + 32 * kSlots; k < r.len; k += 32) {
        const int cc = kDense ? k : ld_stream(P.col_idx + r.start + k);
        const float av = to_f32(ld_stream(vals + r.start + k));
        const float4 sv = ld_state(state + cc * stride);
        const float dx = -gamma * fmaf(delta, av, sv.z * fmaf(lambda, sv.x, sv.y));
        red_add_v2(P.state + cc * stride, dx, delta * av * inv_n);
    }
    if (lane == 0) red_add_f32(P.alpha + i, delta);
}

// One warp's share of a launch: updates warp, warp + W, warp + 2W, ... of P.
template <typename T, bool kDense>
__device__ __forceinline__ void warp_updates(const UpdateParams &P, int warp, int lane) {
    const T *__restrict__ vals = static_cast<const T *>(P.values);
    const int64_t W = P.nwarps;

    uint64_t deadline = 0;
    if (P.deadline_ns) {  // budget relative to this warp's start (warp-uniform)
        const uint64_t now = __shfl_sync(kFull, globaltimer_ns(), 0);
        deadline = now + P.deadline_ns;
    }
    bool bad = false;
    // Software pipeline over this warp's rows with four register buffers
    // whose roles rotate by unrolling (no buffer is ever copied, so no copy
    // waits on a load in flight): in each step the row in X is processed,
    // Y's CSR slice is in flight since the previous step, Z's slice is
    // requested (its row_ptr entries arrived during the previous step) and
    // V's row_ptr entries are requested.
    int64_t t = warp;
    RowData rA, rB, rC, rD;
    int64_t iA = row_of(P, t, bad);
    int64_t iB = iA >= 0 ? row_of(P, t + W, bad) : -1;
    int64_t iC = iB >= 0 ? row_of(P, t + 2 * W, bad) : -1;
    int64_t iD = -1;
    if (iA >= 0) load_meta<kDense>(P, iA, rA);
    if (iB >= 0) load_meta<kDense>(P, iB, rB);
    if (iC >= 0) load_meta<kDense>(P, iC, rC);
    if (iA >= 0) load_slots<T, kDense>(P, vals, rA, lane);
    if (iB >= 0) load_slots<T, kDense>(P, vals, rB, lane);
    int64_t done = 0;
    bool stop = false;
    auto step = [&](int64_t iX, const RowData &X, int64_t iZ, RowData &Z, int64_t &iV, RowData &V) {
        if (iZ >= 0) load_slots<T, kDense>(P, vals, Z, lane);
        iV = iZ >= 0 ? row_of(P, t + 3 * W, bad) : -1;
        if (iV >= 0) load_meta<kDense>(P, iV, V);
        process_row<T, kDense>(P, vals, iX, X, lane);
        if (P.fence_each) {
            __threadfence();
            __syncwarp();
        }
        if (deadline && ((++done & 31) == 0)) {
            const uint64_t now = __shfl_sync(kFull, globaltimer_ns(), 0);
            if (now > deadline) {
                if (lane == 0) atomicOr(P.status, 1);
                stop = true;
            }
        }
        t += W;
    };
#pragma unroll 1
    while (true) {
        if (iA < 0 || stop) break;
        step(iA, rA, iC, rC, iD, rD);
        if (iB < 0 || stop) break;
        step(iB, rB, iD, rD, iA, rA);
        if (iC < 0 || stop) break;
        step(iC, rC, iA, rA, iB, rB);
        if (iD < 0 || stop) break;
        step(iD, rD, iB, rB, iC, rC);
    }
    if (stop) return;
    if (bad && lane == 0) atomicOr(P.status, 2);
}

template <typename T, bool kDense>
__global__ void __launch_bounds__(kUpdateBlock, 2) update_kernel(const UpdateParams P) {
    const int lane = threadIdx.x & 31;
    const int warp = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
    if (warp >= P.nwarps) return;
    warp_updates<T, kDense>(P, warp, lane);
}

// Many independent problems in one launch: block b serves instance
// inst = the last i with block_begin[i] <= b, whose parameters are copied to
// shared memory once; its warps split that instance's updates.
template <typename T, bool kDense>
__global__ void __launch_bounds__(kBatchBlock) batch_update_kernel(const UpdateParams *__restrict__ params,
                                                                   const int *__restrict__ block_begin, int count) {
    __shared__ UpdateParams sp;
    __shared__ int s_inst;
    if (threadIdx.x == 0) {
        int lo = 0, hi = count - 1;  // binary search: last instance whose first block <= blockIdx.x
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (block_begin[mid] <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
        }
        s_inst = lo;
        sp = params[lo];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int warp = (int)(((blockIdx.x - block_begin[s_inst]) * (unsigned)blockDim.x + threadIdx.x) >> 5);
    if (warp >= sp.nwarps || sp.count <= 0) return;
    warp_updates<T, kDense>(sp, warp, lane);
}

template <typename T, bool kDense>
static cudaError_t launch_t(const UpdateParams &p, int grid, int block, cudaStream_t s) {
    update_kernel<T, kDense><<<grid, block, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_update(const UpdateParams &p, int vtype, bool dense, int grid, int block,
                          cudaStream_t s) {
    switch (vtype) {
    case kF32: return dense ? launch_t<float, true>(p, grid, block, s) : launch_t<float, false>(p, grid, block, s);
    case kBF16:
        return dense ? launch_t<__nv_bfloat16, true>(p, grid, block, s)
                     : launch_t<__nv_bfloat16, false>(p, grid, block, s);
    case kF16: return dense ? launch_t<__half, true>(p, grid, block, s) : launch_t<__half, false>(p, grid, block, s);
    default: return cudaErrorInvalidValue;
    }
}

template <typename T, bool kDense>
static cudaError_t batch_launch_t(const UpdateParams *params, const int *block_begin, int count, int grid,
                                  cudaStream_t s) {
    batch_update_kernel<T, kDense><<<grid, kBatchBlock, 0, s>>>(params, block_begin, count);
    return cudaGetLastError();
}

cudaError_t launch_batch_update(const UpdateParams *params, const int *block_begin, int count, int grid, int vtype,
                                bool dense, cudaStream_t s) {
    switch (vtype) {
    case kF32:
        return dense ? batch_launch_t<float, true>(params, block_begin, count, grid, s)
                     : batch_launch_t<float, false>(params, block_begin, count, grid, s);
    case kBF16:
        return dense ? batch_launch_t<__nv_bfloat16, true>(params, block_begin, count, grid, s)
                     : batch_launch_t<__nv_bfloat16, false>(params, block_begin, count, grid, s);
    case kF16:
        return dense ? batch_launch_t<__half, true>(params, block_begin, count, grid, s)
                     : batch_launch_t<__half, false>(params, block_begin, count, grid, s);
    default: return cudaErrorInvalidValue;
    }
}

template <typename T, bool kDense>
static int batch_occ() {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_update_kernel<T, kDense>, kBatchBlock, 0) !=
        cudaSuccess)
        return 1;
    return nb > 0 ? nb : 1;
}

int batch_update_max_blocks_per_sm(int vtype, bool dense) {
    switch (vtype) {
    case kF32: return dense ? batch_occ<float, true>() : batch_occ<float, false>();
    case kBF16: return dense ? batch_occ<__nv_bfloat16, true>() : batch_occ<__nv_bfloat16, false>();
    case kF16: return dense ? batch_occ<__half, true>() : batch_occ<__half, false>();
    default: return 1;
    }
}

template <typename T, bool kDense>
static int occ() {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, update_kernel<T, kDense>, kUpdateBlock, 0) !=
        cudaSuccess)
        return 1;
    return nb > 0 ? nb : 1;
}

int update_max_blocks_per_sm(int vtype, bool dense) {
    switch (vtype) {
    case kF32: return dense ? occ<float, true>() : occ<float, false>();
    case kBF16: return dense ? occ<__nv_bfloat16, true>() : occ<__nv_bfloat16, false>();
    case kF16: return dense ? occ<__half, true>() : occ<__half, false>();
    default: return 1;
    }
}

}  // namespace asaga
