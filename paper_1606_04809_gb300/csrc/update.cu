// The asynchronous Sparse SAGA update kernel (Algorithm 2 of arXiv:1606.04809
// with the projected l2 term of Sec. 4.2).
//
// Each warp is one ASAGA "core".  Update t of a launch samples its row
// i = sample_row(seed, t) before reading anything (Algorithm 2: sample, then
// read), reads x^ and abar on S_i inconsistently (other warps keep adding to
// them), forms delta = phi'_i(a_i.x^) - alpha_i, and applies
//     x_v += -gamma (delta a_iv + D_v (abar_v + lambda x^_v)),
//     abar_v += delta a_iv / n,           for v in S_i,
// as one vector atomic add per column at L2.  The memory alpha_i is swapped
// atomically (atomicExch) and delta is taken against the value it replaced,
// so abar = (1/n) sum_i alpha_i a_i holds in exact arithmetic even when two
// warps visit the same row at once.
//
// Layout: A in CSR (int64 row_ptr, int32 col_idx, values in fp32/bf16/fp16)
// or dense row-major; per-column state float4 {x, abar, D, 0} so that one
// 16-byte L2 read serves x^_v, abar_v and D_v.  Row elements are spread over
// the 32 lanes; up to 32 * kSlots elements stay in registers between the
// dot product and the scatter; the rest of a longer row is read again.
#include "asaga_internal.h"
#include "device_common.cuh"

namespace asaga {

constexpr int kSlots = 4;

template <typename T, bool kDense>
__device__ __forceinline__ void update_row(const UpdateParams &P, const T *__restrict__ vals, int64_t i,
                                           int lane) {
    int64_t start;
    int len;
    if (kDense) {
        start = i * P.d;
        len = (int)P.d;
    } else {
        start = __ldg(P.row_ptr + i);
        len = (int)(__ldg(P.row_ptr + i + 1) - start);
    }
    const float b = __ldg(P.labels + i);
    const float4 *__restrict__ state = P.state;
    const int64_t stride = P.stride;

    int c[kSlots];
    float a[kSlots];
    float4 s[kSlots];
#pragma unroll
    for (int r = 0; r < kSlots; ++r) {
        const int k = lane + 32 * r;
        c[r] = 0;
        a[r] = 0.f;
        if (k < len) {
            c[r] = kDense ? k : ld_stream(P.col_idx + start + k);
            a[r] = to_f32(ld_stream(vals + start + k));
        }
    }
    float z = 0.f;
#pragma unroll
    for (int r = 0; r < kSlots; ++r) {
        const int k = lane + 32 * r;
        s[r] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (k < len) s[r] = ld_state(state + c[r] * stride);
    }
#pragma unroll
    for (int r = 0; r < kSlots; ++r) z = fmaf(a[r], s[r].x, z);
    for (int k = lane + 32 * kSlots; k < len; k += 32) {  // rest of a long row
        const int cc = kDense ? k : ld_stream(P.col_idx + start + k);
        z = fmaf(to_f32(ld_stream(vals + start + k)), ld_state(state + cc * stride).x, z);
    }
    z = warp_sum(z);

    float delta = 0.f;
    if (lane == 0) {
        const float g = phi_prime_f32(P.loss, z, b);
        const float old = atomicExch(P.alpha + i, g);
        delta = g - old;
    }
    delta = __shfl_sync(kFull, delta, 0);

    const float gamma = P.gamma, lambda = P.lambda, inv_n = P.inv_n;
#pragma unroll
    for (int r = 0; r < kSlots; ++r) {
        const int k = lane + 32 * r;
        if (k < len) {
            const float dx = -gamma * fmaf(delta, a[r], s[r].z * fmaf(lambda, s[r].x, s[r].y));
            red_add_v2(P.state + c[r] * stride, dx, delta * a[r] * inv_n);
        }
    }
    for (int k = lane + 32 * kSlots; k < len; k += 32) {
        const int cc = kDense ? k : ld_stream(P.col_idx + start + k);
        const float av = to_f32(ld_stream(vals + start + k));
        const float4 sv = ld_state(state + cc * stride);
        const float dx = -gamma * fmaf(delta, av, sv.z * fmaf(lambda, sv.x, sv.y));
        red_add_v2(P.state + cc * stride, dx, delta * av * inv_n);
    }
}

template <typename T, bool kDense>
__global__ void __launch_bounds__(kUpdateBlock, 4) update_kernel(const UpdateParams P) {
    const int lane = threadIdx.x & 31;
    const int warp = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
    if (warp >= P.nwarps) return;
    const T *__restrict__ vals = static_cast<const T *>(P.values);

    uint64_t deadline = 0;
    if (P.deadline_ns) {  // budget relative to this warp's start (warp-uniform)
        uint64_t now = __shfl_sync(kFull, globaltimer_ns(), 0);
        deadline = now + P.deadline_ns;
    }
    int64_t done = 0;
    for (int64_t t = warp; t < P.count; t += P.nwarps) {
        int64_t i;
        if (P.idx) {
            i = __ldg(P.idx + t);
            if (i < 0 || i >= P.n) {
                if (lane == 0) atomicOr(P.status, 2);
                return;
            }
        } else {
            i = sample_row(P.seed, P.t_begin + (uint64_t)t, P.n);
        }
        update_row<T, kDense>(P, vals, i, lane);
        if (P.fence_each) {
            __threadfence();
            __syncwarp();
        }
        if (deadline && ((++done & 63) == 0)) {
            const uint64_t now = __shfl_sync(kFull, globaltimer_ns(), 0);
            if (now > deadline) {
                if (lane == 0) atomicOr(P.status, 1);
                return;
            }
        }
    }
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
