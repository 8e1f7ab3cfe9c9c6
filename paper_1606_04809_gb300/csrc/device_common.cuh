// Device helpers shared by the solver's kernels.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "asaga_internal.h"

namespace asaga {

constexpr unsigned kFull = 0xffffffffu;

template <typename T> __device__ __forceinline__ float to_f32(T v);
template <> __device__ __forceinline__ float to_f32<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f32<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <> __device__ __forceinline__ float to_f32<__half>(__half v) { return __half2float(v); }

// Streaming read of A (each row is read once per visit; evict-first so that
// the solver state keeps the L2).
template <typename T> __device__ __forceinline__ T ld_stream(const T *p) { return __ldcs(p); }

// ---- layouts of A in the steady-state kernels --------------------------
// Values: float / bf16 / half per entry, or RowScale (one float per row).
// Column indices: int32_t or uint16_t (d <= 65536).
struct RowScale {};
template <typename T> struct IsRowScale { static constexpr bool value = false; };
template <> struct IsRowScale<RowScale> { static constexpr bool value = true; };

// Column index of entry k, read-only path / streaming path.
template <typename I> __device__ __forceinline__ int col_ro(const void *col, int64_t k) {
    return (int)__ldg(static_cast<const I *>(col) + k);
}
template <typename I> __device__ __forceinline__ int col_stream(const void *col, int64_t k) {
    return (int)__ldcs(static_cast<const I *>(col) + k);
}
// Value of entry k of row i.
template <typename T> __device__ __forceinline__ float value_at(const void *values, int64_t i, int64_t k) {
    if constexpr (IsRowScale<T>::value)
        return static_cast<const float *>(values)[i];
    else
        return to_f32(static_cast<const T *>(values)[k]);
}

// Calls f.template run<T, I, kDense>() for a layout (ValType | kIdx16);
// returns `bad` for a layout without kernels.
template <typename R, typename F> R with_layout(int layout, bool dense, F &&f, R bad) {
    const int v = layout & ~kIdx16;
    if (dense) {
        switch (v) {
        case kF32: return f.template run<float, int32_t, true>();
        case kBF16: return f.template run<__nv_bfloat16, int32_t, true>();
        case kF16: return f.template run<__half, int32_t, true>();
        default: return bad;
        }
    }
    if (layout & kIdx16) {
        switch (v) {
        case kF32: return f.template run<float, uint16_t, false>();
        case kBF16: return f.template run<__nv_bfloat16, uint16_t, false>();
        case kF16: return f.template run<__half, uint16_t, false>();
        case kRowScale: return f.template run<RowScale, uint16_t, false>();
        default: return bad;
        }
    }
    switch (v) {
    case kF32: return f.template run<float, int32_t, false>();
    case kBF16: return f.template run<__nv_bfloat16, int32_t, false>();
    case kF16: return f.template run<__half, int32_t, false>();
    case kRowScale: return f.template run<RowScale, int32_t, false>();
    default: return bad;
    }
}

// Read of shared state at L2 (bypasses L1, which is not coherent with the
// atomics other SMs apply).
__device__ __forceinline__ float2 ld_state(const float2 *p) { return __ldcg(p); }

// Read of state that no thread writes during the kernel (evaluations), and
// of the constant D: L1-cached, non-coherent path.
__device__ __forceinline__ float2 ld_state_ro(const float2 *p) { return __ldg(p); }
__device__ __forceinline__ float ld_d(const float *p) { return __ldg(p); }

// x_v += dx and abar_v += dab as one vector reduction at L2 (each element
// is added atomically; nothing is returned).
__device__ __forceinline__ void red_add_v2(float2 *p, float dx, float dab) {
    asm volatile("red.relaxed.gpu.global.add.v2.f32 [%0], {%1, %2};" ::"l"(p), "f"(dx), "f"(dab)
                 : "memory");
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(kFull, v, o));
    return v;
}

// The output mix of SplitMix64 (Steele, Lea and Flood, OOPSLA 2014).
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// SplitMix64 used as a counter-based generator: output number t+1 of the
// stream seeded with `seed` (its state advances by the golden gamma).
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t t) {
    return mix64(seed + (t + 1) * 0x9E3779B97F4A7C15ull);
}

// Row index of update t: uniform in [0, n) with replacement (Algorithm 2
// samples i before reading anything), by multiply-high range reduction.
__device__ __forceinline__ int64_t sample_row(uint64_t seed, uint64_t t, int64_t n) {
    return (int64_t)__umul64hi(splitmix64_at(seed, t), (uint64_t)n);
}

// Row index of update t when every epoch visits each row once: position
// p = t mod n of epoch e = t / n goes through a 4-round balanced Feistel
// network on 2h bits (4^h >= n) keyed by the epoch, and the network is
// applied again until the value falls below n (cycle walking).  The network
// is a bijection of [0, 4^h), so the walk from p < n reaches a value below n
// within p's cycle; the iteration cap is never reached in practice (each
// step lands below n with probability >= 1/4) and only keeps the loop bounded.
__device__ __forceinline__ int64_t permuted_row(uint64_t seed, uint64_t t, int64_t n) {
    constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ull;
    const uint64_t nn = (uint64_t)n;
    const uint64_t e = t / nn, pos = t - e * nn;
    const int bits = nn > 1 ? 64 - __clzll((long long)(nn - 1)) : 0;
    const int h = bits > 1 ? (bits + 1) / 2 : 1;
    const uint64_t mask = (1ull << h) - 1;
    const uint64_t key = splitmix64_at(seed ^ 0xD1B54A32D192ED03ull, e);
    uint64_t x = pos;
    for (int walk = 0; walk < 4096; ++walk) {
        uint64_t L = x >> h, R = x & mask;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const uint64_t f = mix64((key ^ R) + (uint64_t)(r + 1) * kGolden) & mask;
            const uint64_t nl = R;
            R = L ^ f;
            L = nl;
        }
        x = (L << h) | R;
        if (x < nn) return (int64_t)x;
    }
    return (int64_t)pos;
}

__device__ __forceinline__ int64_t sampled_row(int sampling, uint64_t seed, uint64_t t, int64_t n) {
    return sampling == 1 ? permuted_row(seed, t, n) : sample_row(seed, t, n);
}

// phi'(z) in float32.  Logistic: -b / (1 + exp(b z)); squared: z - y.
// exp(-|t|) lies in (0, 1], where CUDA's fast __expf is within a few ulp;
// the division uses the correctly rounded reciprocal.
__device__ __forceinline__ float phi_prime_f32(int loss, float z, float b) {
    if (loss == 0) {
        const float t = b * z;
        const float e = __expf(-fabsf(t));     // in (0, 1]
        const float r = __frcp_rn(1.f + e);    // 1 / (1 + e)
        const float s = (t >= 0.f) ? e * r : r;  // 1 / (1 + exp(t))
        return -b * s;
    }
    return z - b;
}

// phi(z) and phi'(z) in float64.
__device__ __forceinline__ double phi_f64(int loss, double z, double b) {
    if (loss == 0) {
        double t = b * z;  // log(1 + exp(-t))
        return fmax(-t, 0.0) + log1p(exp(-fabs(t)));
    }
    double r = z - b;
    return 0.5 * r * r;
}

__device__ __forceinline__ double phi_prime_f64(int loss, double z, double b) {
    if (loss == 0) {
        double t = b * z;
        double e = exp(-fabs(t));
        double s = (t >= 0.0) ? e / (1.0 + e) : 1.0 / (1.0 + e);
        return -b * s;
    }
    return z - b;
}

}  // namespace asaga
