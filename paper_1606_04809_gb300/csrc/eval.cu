// Float64 evaluation and set-up kernels of the ASAGA solver.
//
//   objective      f(x) = 1/n sum_i phi_i(a_i.x) + lambda/2 |x|^2  (Eq. finiteSum, Sec. 4.1)
//   gradient       1/n A^T phi'(A x) + lambda x
//   abar recompute abar = 1/n sum_i alpha_i a_i  (Sec. 2, definition of abar)
//   set-up         column counts -> D_v = n / |{i : v in S_i}| (Sec. 2),
//                  L = max_i (c |a_i|^2 + lambda max_{v in S_i} D_v),
//                  value conversion to the storage type.
//
// One thread evaluates one row (grid-stride over rows), so the float64
// phi of 32 rows runs as one warp instruction.  Row sums a_i . x are
// compensated float32 sums (about 48 significant bits) of the float32
// state and stored values, widened to float64 per row; everything after
// that (phi, row totals, column sums) is float64.  Nothing writes the state
// while these kernels run, so x is read through the L1-cached read-only
// path: the most frequent columns, which appear in nearly every row, are
// served by each SM's L1 instead of serialising at one L2 line.  Block
// results go to a partial array reduced by one block in a fixed order, so
// objective values are bitwise reproducible.  Column scatters (A^T w) use
// float64 atomics at L2; dense problems with few columns, and the most
// frequent columns of sparse ones, first accumulate per block in shared
// memory.
#include <algorithm>

#include "asaga_internal.h"
#include "device_common.cuh"

namespace asaga {

constexpr int kSmemCols = 2048;  // dense problems up to this d accumulate per block in shared memory

// Compensated ("float-float") accumulation of a_k x_k: each product is split
// exactly into p + e with an FMA (Dekker/Ogita-Rump-Oishi TwoProduct) and
// summed with Knuth's TwoSum into a (hi, lo) pair, giving about 48
// significant bits on the fast float32 pipe.  GB300's float64 pipe is a
// small fraction of its float32 rate, so the per-entry work stays in float32
// and only per-row results are widened to float64.
struct FF {
    float hi = 0.f, lo = 0.f;
};
__device__ __forceinline__ void ff_add_product(FF &acc, float a, float b) {
    const float p = __fmul_rn(a, b);
    const float e = __fmaf_rn(a, b, -p);
    const float s = __fadd_rn(acc.hi, p);
    const float bb = __fsub_rn(s, acc.hi);
    const float err = __fadd_rn(__fsub_rn(acc.hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    acc.hi = s;
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(err, e));
}
__device__ __forceinline__ double ff_value(const FF &a) { return (double)a.hi + (double)a.lo; }

// z_i = a_i . x for one row, by one thread (rows are split over threads so
// that the float64 work per row runs on all 32 lanes at once).
template <typename T, typename I>
__device__ __forceinline__ double row_dot_thread(const EvalParams &P, int64_t i, int64_t start, int len, bool dense) {
    FF acc;
#pragma unroll 4
    for (int k = 0; k < len; ++k) {
        const int c = dense ? k : col_ro<I>(P.col_idx, start + k);
        ff_add_product(acc, value_at<T>(P.values, i, start + k), ld_state_ro(P.state + (int64_t)c * P.stride).x);
    }
    return ff_value(acc);
}

template <typename T, bool kDense>
__device__ __forceinline__ void row_range(const EvalParams &P, int64_t i, int64_t &start, int &len) {
    if (kDense) {
        start = i * P.d;
        len = (int)P.d;
    } else {
        start = P.row_ptr[i];
        len = (int)(P.row_ptr[i + 1] - start);
    }
}

// Deterministic block reduction (sum or max) of one double per thread.
__device__ __forceinline__ double block_reduce(double v, bool is_max) {
    __shared__ double red[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    v = is_max ? warp_max(v) : warp_sum(v);
    if (lane == 0) red[w] = v;
    __syncthreads();
    const int nw = blockDim.x >> 5;
    double r = 0.0;
    if (w == 0) {
        r = lane < nw ? red[lane] : 0.0;
        r = is_max ? warp_max(r) : warp_sum(r);
    }
    __syncthreads();
    return r;  // valid in thread 0
}

template <typename T, typename I, bool kDense>
__global__ void __launch_bounds__(kEvalBlock) objective_rows_kernel(const EvalParams P, double *partial) {
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P.n; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t start;
        int len;
        row_range<T, kDense>(P, i, start, len);
        const double z = row_dot_thread<T, I>(P, i, start, len, kDense);
        acc += phi_f64(P.loss, z, P.labels[i]);
    }
    double xx = 0.0;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < P.d; v += (int64_t)gridDim.x * blockDim.x) {
        const double xv = ld_state_ro(P.state + v * P.stride).x;
        xx += xv * xv;
    }
    const double s1 = block_reduce(acc, false);
    const double s2 = block_reduce(xx, false);
    if (threadIdx.x == 0) {
        partial[blockIdx.x] = s1;
        partial[gridDim.x + blockIdx.x] = s2;
    }
}

// The objective of many instances in one launch: blockIdx.y = instance,
// blockIdx.x = one of gridDim.x blocks over that instance's rows.
template <typename T, typename I, bool kDense>
__global__ void __launch_bounds__(kEvalBlock) batch_objective_rows_kernel(const EvalParams *__restrict__ params,
                                                                          double *partial) {
    __shared__ EvalParams sp;
    if (threadIdx.x == 0) sp = params[blockIdx.y];
    __syncthreads();
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < sp.n; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t start;
        int len;
        row_range<T, kDense>(sp, i, start, len);
        acc += phi_f64(sp.loss, row_dot_thread<T, I>(sp, i, start, len, kDense), sp.labels[i]);
    }
    double xx = 0.0;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < sp.d; v += (int64_t)gridDim.x * blockDim.x) {
        const double xv = ld_state_ro(sp.state + v * sp.stride).x;
        xx += xv * xv;
    }
    const double s1 = block_reduce(acc, false);
    const double s2 = block_reduce(xx, false);
    if (threadIdx.x == 0) {
        double *p = partial + 2 * ((int64_t)blockIdx.y * gridDim.x + blockIdx.x);
        p[0] = s1;
        p[1] = s2;
    }
}

// f_out[i] <- (sum of instance i's row partials)/n_i + lambda_i/2 (sum of its x partials); one block per instance.
__global__ void batch_objective_finish_kernel(const EvalParams *__restrict__ params, const double *partial, int grid,
                                              double *f_out) {
    const double *p = partial + 2 * (int64_t)blockIdx.x * grid;
    double a = 0.0, b = 0.0;
    for (int j = threadIdx.x; j < grid; j += blockDim.x) {
        a += p[2 * j];
        b += p[2 * j + 1];
    }
    const double sa = block_reduce(a, false);
    const double sb = block_reduce(b, false);
    if (threadIdx.x == 0) {
        const EvalParams &e = params[blockIdx.x];
        f_out[blockIdx.x] = sa / (double)e.n + 0.5 * e.lambda * sb;
    }
}

__global__ void objective_finish_kernel(const double *partial, int grid, double inv_n, double lambda,
                                        double *out) {
    double a = 0.0, b = 0.0;
    for (int j = threadIdx.x; j < grid; j += blockDim.x) {
        a += partial[j];
        b += partial[grid + j];
    }
    const double sa = block_reduce(a, false);
    const double sb = block_reduce(b, false);
    if (threadIdx.x == 0) out[0] = sa * inv_n + 0.5 * lambda * sb;
}

// acc[v] += sum_i w_i a_iv, w_i = phi'_i(a_i.x)/n (mode 0) or alpha_i/n (mode 1).
// kSlots: 0 = every column goes straight to a float64 atomic at L2;
//         1 = dense rows, all d columns accumulate per block in shared memory;
//         2 = the n_hot most frequent columns accumulate per block in shared
//             memory (their atomics would otherwise serialise at one L2 line).
template <typename T, typename I, bool kDense, int kSlotsMode>
__global__ void __launch_bounds__(kEvalBlock) scatter_rows_kernel(const EvalParams P, int mode, double *acc) {
    extern __shared__ double sacc[];
    const double inv_n = 1.0 / (double)P.n;
    const int nslots = kSlotsMode == 1 ? (int)P.d : (kSlotsMode == 2 ? P.n_hot : 0);
    if (kSlotsMode) {
        for (int v = threadIdx.x; v < nslots; v += blockDim.x) sacc[v] = 0.0;
        __syncthreads();
    }
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P.n; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t start;
        int len;
        row_range<T, kDense>(P, i, start, len);
        double w;
        if (mode == 0) {
            const double z = row_dot_thread<T, I>(P, i, start, len, kDense);
            w = phi_prime_f64(P.loss, z, P.labels[i]) * inv_n;
        } else {
            w = (double)P.alpha[i] * inv_n;
        }
#pragma unroll 4
        for (int k = 0; k < len; ++k) {
            const int c = kDense ? k : col_ro<I>(P.col_idx, start + k);
            const double contrib = w * (double)value_at<T>(P.values, i, start + k);
            const int slot = kSlotsMode == 1 ? c : (kSlotsMode == 2 ? __ldg(P.hot_slot + c) : -1);
            if (slot >= 0)
                atomicAdd(sacc + slot, contrib);
            else
                atomicAdd(acc + c, contrib);
        }
    }
    if (kSlotsMode) {
        __syncthreads();
        for (int v = threadIdx.x; v < nslots; v += blockDim.x)
            atomicAdd(acc + (kSlotsMode == 1 ? v : P.hot_col[v]), sacc[v]);
    }
}

// The abar recomputation: acc[v] += sum_i (alpha_i/n) a_iv.  A row's weight
// is one load, so a warp takes a row and its lanes split the entries
// (coalesced loads of the CSR streams, unlike one thread per row, which
// mode 0 needs for its float64 phi'); the frequent columns (kSlotsMode 2) or
// all d dense columns (kSlotsMode 1) accumulate per block in shared memory
// as in scatter_rows_kernel.  Rows with alpha_i = 0 add nothing and are
// skipped.
template <typename T, typename I, bool kDense, int kSlotsMode>
__global__ void __launch_bounds__(kEvalBlock) scatter_alpha_rows_kernel(const EvalParams P, double *acc) {
    extern __shared__ double sacc[];
    const double inv_n = 1.0 / (double)P.n;
    const int nslots = kSlotsMode == 1 ? (int)P.d : (kSlotsMode == 2 ? P.n_hot : 0);
    if (kSlotsMode) {
        for (int v = threadIdx.x; v < nslots; v += blockDim.x) sacc[v] = 0.0;
        __syncthreads();
    }
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp; i < P.n; i += nwarps) {
        const double w = (double)__ldg(P.alpha + i) * inv_n;  // the same in every lane
        if (w == 0.0) continue;
        int64_t start;
        int len;
        row_range<T, kDense>(P, i, start, len);
        for (int k = lane; k < len; k += 32) {
            const int c = kDense ? k : col_stream<I>(P.col_idx, start + k);
            const double contrib = w * (double)value_at<T>(P.values, i, start + k);
            const int slot = kSlotsMode == 1 ? c : (kSlotsMode == 2 ? __ldg(P.hot_slot + c) : -1);
            if (slot >= 0)
                atomicAdd(sacc + slot, contrib);
            else
                atomicAdd(acc + c, contrib);
        }
    }
    if (kSlotsMode) {
        __syncthreads();
        for (int v = threadIdx.x; v < nslots; v += blockDim.x)
            atomicAdd(acc + (kSlotsMode == 1 ? v : P.hot_col[v]), sacc[v]);
    }
}

// ---- the batched abar recomputation (blockIdx.y = instance)

__global__ void __launch_bounds__(kEvalBlock) batch_zero_acc_kernel(const EvalParams *__restrict__ params) {
    const EvalParams &e = params[blockIdx.y];
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < e.d; v += (int64_t)gridDim.x * blockDim.x)
        e.acc[v] = 0.0;
}

// acc_i[v] += sum_r (alpha_r / n_i) a_rv over instance i's rows, a warp per
// row; the instance's frequent columns (or all of its dense columns, up to
// kSmemCols) accumulate per block in shared memory first.
template <typename T, typename I, bool kDense>
__global__ void __launch_bounds__(kEvalBlock) batch_scatter_alpha_kernel(const EvalParams *__restrict__ params) {
    extern __shared__ double sacc[];
    __shared__ EvalParams sp;
    if (threadIdx.x == 0) sp = params[blockIdx.y];
    __syncthreads();
    if (sp.n <= 0) return;
    const int nslots = kDense ? (sp.d <= kSmemCols ? (int)sp.d : 0) : (sp.hot_slot ? sp.n_hot : 0);
    for (int v = threadIdx.x; v < nslots; v += blockDim.x) sacc[v] = 0.0;
    __syncthreads();
    const double inv_n = 1.0 / (double)sp.n;
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp; i < sp.n; i += nwarps) {
        const double w = (double)__ldg(sp.alpha + i) * inv_n;  // the same in every lane
        if (w == 0.0) continue;
        int64_t start;
        int len;
        row_range<T, kDense>(sp, i, start, len);
        for (int k = lane; k < len; k += 32) {
            const int c = kDense ? k : col_stream<I>(sp.col_idx, start + k);
            const double contrib = w * (double)value_at<T>(sp.values, i, start + k);
            const int slot = kDense ? (nslots ? c : -1) : (nslots ? __ldg(sp.hot_slot + c) : -1);
            if (slot >= 0)
                atomicAdd(sacc + slot, contrib);
            else
                atomicAdd(sp.acc + c, contrib);
        }
    }
    __syncthreads();
    for (int v = threadIdx.x; v < nslots; v += blockDim.x)
        atomicAdd(sp.acc + (kDense ? v : sp.hot_col[v]), sacc[v]);
}

// abar_v <- (float)acc_v over instance i's columns; partial[i * grid + b] <-
// the block's max |abar_v(before) - acc_v|.
__global__ void __launch_bounds__(kEvalBlock) batch_abar_finish_kernel(const EvalParams *__restrict__ params,
                                                                       double *partial) {
    const EvalParams &e = params[blockIdx.y];
    double local = 0.0;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < e.d; v += (int64_t)gridDim.x * blockDim.x) {
        float2 *sv = e.state + v * e.stride;
        const double exact = e.acc[v];
        local = fmax(local, fabs((double)sv->y - exact));
        sv->y = (float)exact;
    }
    const double r = block_reduce(local, true);
    if (threadIdx.x == 0) partial[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = r;
}

__global__ void batch_drift_kernel(const double *partial, int grid, double *drift_out) {
    const double *p = partial + (int64_t)blockIdx.x * grid;
    double v = 0.0;
    for (int j = threadIdx.x; j < grid; j += blockDim.x) v = fmax(v, p[j]);
    const double r = block_reduce(v, true);
    if (threadIdx.x == 0) drift_out[blockIdx.x] = r;
}

__global__ void __launch_bounds__(kEvalBlock) column_finish_kernel(const EvalParams P, int mode, double *acc,
                                                                   double *partial) {
    double local = 0.0;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < P.d; v += (int64_t)gridDim.x * blockDim.x) {
        float2 *sp = P.state + v * P.stride;
        if (mode == 0) {
            const double g = acc[v] + P.lambda * (double)sp->x;
            acc[v] = g;
            local += g * g;
        } else {
            const double exact = acc[v];
            local = fmax(local, fabs((double)sp->y - exact));
            sp->y = (float)exact;
        }
    }
    const double r = block_reduce(local, mode == 1);
    if (threadIdx.x == 0) partial[blockIdx.x] = r;
}

__global__ void reduce_partials_kernel(const double *partial, int grid, int mode, double *out) {
    double v = 0.0;
    for (int j = threadIdx.x; j < grid; j += blockDim.x) v = mode == 1 ? fmax(v, partial[j]) : v + partial[j];
    const double r = block_reduce(v, mode == 1);
    if (threadIdx.x == 0) out[0] = r;
}

// ------------------------------------------------------------------ set-up

// Column counts.  A column in most rows would take one global atomic per
// row on a single address; instead each block counts into a shared-memory
// open-addressing table (kCountSlots slots, 4 linear probes, a slot's key is
// written once) and adds its totals to global memory at the end.  An entry
// whose probes all hold other columns goes straight to global memory.
// Columns outside [0, d) are skipped: the kernel runs while the host is still
// checking the problem.
constexpr int kCountSlots = 4096;
constexpr int kCountBlocks = 1216;  // 152 SMs x 8 blocks of 256 threads
__global__ void __launch_bounds__(256) count_columns_kernel(const int32_t *col, int64_t nnz, int64_t d, int *count) {
    __shared__ int key[kCountSlots];
    __shared__ int cnt[kCountSlots];
    for (int j = threadIdx.x; j < kCountSlots; j += blockDim.x) {
        key[j] = -1;
        cnt[j] = 0;
    }
    __syncthreads();
    volatile int *vkey = key;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz; k += (int64_t)gridDim.x * blockDim.x) {
        const int c = col[k];
        if (c < 0 || c >= d) continue;
        const unsigned h = ((unsigned)c * 2654435761u) >> 20;  // 12 bits (Knuth's multiplicative hash)
        bool done = false;
        for (int probe = 0; probe < 4 && !done; ++probe) {
            const int slot = (int)((h + probe) & (kCountSlots - 1));
            int kv = vkey[slot];
            if (kv == -1) kv = atomicCAS(&key[slot], -1, c);  // the key before this thread's attempt
            if (kv == -1 || kv == c) {
                atomicAdd(&cnt[slot], 1);
                done = true;
            }
        }
        if (!done) atomicAdd(count + c, 1);
    }
    __syncthreads();
    for (int j = threadIdx.x; j < kCountSlots; j += blockDim.x)
        if (key[j] >= 0 && cnt[j] > 0) atomicAdd(count + key[j], cnt[j]);
}

__global__ void init_state_kernel(float2 *state, float *dcol, int stride, int64_t d, const int *count, int64_t n) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < d; v += (int64_t)gridDim.x * blockDim.x) {
        float D = 1.f;
        if (count) D = count[v] > 0 ? (float)((double)n / (double)count[v]) : 0.f;
        state[v * stride] = make_float2(0.f, 0.f);
        dcol[v] = D;
    }
}

// Per row: c |a_i|^2 + lambda max_{v in S_i} D_v (the smoothness constant of
// the component the sparse update samples, with the projected l2 term);
// partial[b] <- the block's maximum.  Rows whose range leaves [0, nnz] and
// columns outside [0, d) are skipped: the kernel runs while the host is still
// checking the problem.
template <typename T, bool kDense>
__global__ void __launch_bounds__(kEvalBlock) row_smoothness_kernel(const EvalParams P, int64_t nnz, double c_loss,
                                                                    double *partial) {
    const T *vals = static_cast<const T *>(P.values);
    const int lane = threadIdx.x & 31;
    const int64_t wpb = blockDim.x >> 5;
    const int64_t gw = blockIdx.x * wpb + (threadIdx.x >> 5);
    const int64_t tw = (int64_t)gridDim.x * wpb;
    double best = 0.0;
    for (int64_t i = gw; i < P.n; i += tw) {
        int64_t start;
        int len;
        if (kDense) {
            start = i * P.d;
            len = (int)P.d;
        } else {
            start = P.row_ptr[i];
            const int64_t end = P.row_ptr[i + 1];
            len = (start < 0 || end < start || end > nnz || end - start > INT32_MAX) ? 0 : (int)(end - start);
        }
        double s = 0.0, dmax = 0.0;
        for (int k = lane; k < len; k += 32) {
            const double a = (double)to_f32(vals[start + k]);
            s += a * a;
            const int c = kDense ? k : static_cast<const int32_t *>(P.col_idx)[start + k];
            if (c < 0 || c >= P.d) continue;
            dmax = fmax(dmax, (double)ld_d(P.dcol + c));
        }
        best = fmax(best, c_loss * warp_sum(s) + P.lambda * warp_max(dmax));
    }
    const double r = block_reduce(best, true);
    if (threadIdx.x == 0) partial[blockIdx.x] = r;
}

template <typename S>
__device__ __forceinline__ double src_to_f64(const S *p, int64_t k);
template <> __device__ __forceinline__ double src_to_f64<double>(const double *p, int64_t k) { return p[k]; }
template <> __device__ __forceinline__ double src_to_f64<float>(const float *p, int64_t k) { return p[k]; }
template <> __device__ __forceinline__ double src_to_f64<__nv_bfloat16>(const __nv_bfloat16 *p, int64_t k) {
    return (double)__bfloat162float(p[k]);
}
template <> __device__ __forceinline__ double src_to_f64<__half>(const __half *p, int64_t k) {
    return (double)__half2float(p[k]);
}

template <typename D>
__device__ __forceinline__ D from_f64(double v);
template <> __device__ __forceinline__ float from_f64<float>(double v) { return (float)v; }
template <> __device__ __forceinline__ __nv_bfloat16 from_f64<__nv_bfloat16>(double v) { return __double2bfloat16(v); }
template <> __device__ __forceinline__ __half from_f64<__half>(double v) { return __double2half(v); }

// Round-to-nearest conversion of the input values to the storage type.
template <typename S, typename D>
__global__ void convert_kernel(const S *src, D *dst, int64_t count) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < count; k += (int64_t)gridDim.x * blockDim.x)
        dst[k] = from_f64<D>(src_to_f64<S>(src, k));
}

__global__ void labels_kernel(const double *l64, float *l32, int64_t n) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        l32[k] = (float)l64[k];
}

// ------------------------------------------------------------------ launchers

static int elementwise_grid(int64_t count) {
    int64_t g = (count + 255) / 256;
    if (g > 8192) g = 8192;
    return g < 1 ? 1 : (int)g;
}

struct ObjectiveRows {
    const EvalParams &p;
    int grid;
    double *partial;
    cudaStream_t s;
    template <typename T, typename I, bool kDense> cudaError_t run() const {
        objective_rows_kernel<T, I, kDense><<<grid, kEvalBlock, 0, s>>>(p, partial);
        return cudaGetLastError();
    }
};

cudaError_t launch_objective_rows(const EvalParams &p, int layout, bool dense, int grid, double *partial,
                                  cudaStream_t s) {
    return with_layout(layout, dense, ObjectiveRows{p, grid, partial, s}, cudaErrorInvalidValue);
}

struct BatchObjective {
    const EvalParams *params;
    int count, grid;
    double *partial;
    cudaStream_t s;
    template <typename T, typename I, bool kDense> cudaError_t run() const {
        batch_objective_rows_kernel<T, I, kDense><<<dim3(grid, count), kEvalBlock, 0, s>>>(params, partial);
        return cudaGetLastError();
    }
};

cudaError_t launch_batch_objective(const EvalParams *params, int count, int grid, int layout, bool dense,
                                   double *partial, double *f_out, cudaStream_t s) {
    cudaError_t e = with_layout(layout, dense, BatchObjective{params, count, grid, partial, s}, cudaErrorInvalidValue);
    if (e != cudaSuccess) return e;
    batch_objective_finish_kernel<<<count, 256, 0, s>>>(params, partial, grid, f_out);
    return cudaGetLastError();
}

struct BatchScatterAlpha {
    const EvalParams *params;
    int count, grid;
    size_t smem;
    cudaStream_t s;
    template <typename T, typename I, bool kDense> cudaError_t run() const {
        batch_scatter_alpha_kernel<T, I, kDense><<<dim3(grid, count), kEvalBlock, smem, s>>>(params);
        return cudaGetLastError();
    }
};

cudaError_t launch_batch_recompute(const EvalParams *params, int count, int grid, int layout, bool dense,
                                   int max_hot, double *partial, double *drift_out, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    batch_zero_acc_kernel<<<dim3(grid, count), kEvalBlock, 0, s>>>(params);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t smem = (size_t)(dense ? kSmemCols : std::max(0, max_hot)) * sizeof(double);
    e = with_layout(layout, dense, BatchScatterAlpha{params, count, grid, smem, s}, cudaErrorInvalidValue);
    if (e != cudaSuccess) return e;
    batch_abar_finish_kernel<<<dim3(grid, count), kEvalBlock, 0, s>>>(params, partial);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    batch_drift_kernel<<<count, 256, 0, s>>>(partial, grid, drift_out);
    return cudaGetLastError();
}

cudaError_t launch_objective_finish(const double *partial, int grid, double inv_n, double lambda, double *out,
                                    cudaStream_t s) {
    objective_finish_kernel<<<1, 256, 0, s>>>(partial, grid, inv_n, lambda, out);
    return cudaGetLastError();
}

struct ScatterRows {
    const EvalParams &p;
    int mode, grid;
    double *acc;
    cudaStream_t s;
    template <typename T, typename I, bool kDense> cudaError_t run() const {
        if (mode == 1) {  // abar from alpha: a warp per row
            if constexpr (kDense) {
                if (p.d <= kSmemCols)
                    scatter_alpha_rows_kernel<T, I, true, 1><<<grid, kEvalBlock, (size_t)p.d * sizeof(double), s>>>(p, acc);
                else
                    scatter_alpha_rows_kernel<T, I, true, 0><<<grid, kEvalBlock, 0, s>>>(p, acc);
            } else {
                if (p.n_hot > 0 && p.hot_slot)
                    scatter_alpha_rows_kernel<T, I, false, 2>
                        <<<grid, kEvalBlock, (size_t)p.n_hot * sizeof(double), s>>>(p, acc);
                else
                    scatter_alpha_rows_kernel<T, I, false, 0><<<grid, kEvalBlock, 0, s>>>(p, acc);
            }
            return cudaGetLastError();
        }
        if (kDense && p.d <= kSmemCols) {
            scatter_rows_kernel<T, I, kDense, 1><<<grid, kEvalBlock, (size_t)p.d * sizeof(double), s>>>(p, mode, acc);
        } else if (!kDense && p.n_hot > 0 && p.hot_slot) {
            scatter_rows_kernel<T, I, kDense, 2><<<grid, kEvalBlock, (size_t)p.n_hot * sizeof(double), s>>>(p, mode,
                                                                                                           acc);
        } else {
            scatter_rows_kernel<T, I, kDense, 0><<<grid, kEvalBlock, 0, s>>>(p, mode, acc);
        }
        return cudaGetLastError();
    }
};

cudaError_t launch_scatter_rows(const EvalParams &p, int layout, bool dense, int mode, int grid, double *acc,
                                cudaStream_t s) {
    return with_layout(layout, dense, ScatterRows{p, mode, grid, acc, s}, cudaErrorInvalidValue);
}

cudaError_t launch_column_finish(const EvalParams &p, int mode, int grid, double *acc, double *partial,
                                 cudaStream_t s) {
    column_finish_kernel<<<grid, kEvalBlock, 0, s>>>(p, mode, acc, partial);
    return cudaGetLastError();
}

cudaError_t launch_reduce_partials(const double *partial, int grid, int mode, double *out, cudaStream_t s) {
    reduce_partials_kernel<<<1, 256, 0, s>>>(partial, grid, mode, out);
    return cudaGetLastError();
}

cudaError_t launch_count_columns(const int32_t *col_idx, int64_t nnz, int64_t d, int *count, cudaStream_t s) {
    if (nnz > 0) {
        const int grid = (int)std::min<int64_t>(kCountBlocks, (nnz + 255) / 256);
        count_columns_kernel<<<grid, 256, 0, s>>>(col_idx, nnz, d, count);
    }
    return cudaGetLastError();
}

cudaError_t launch_init_state(float2 *state, float *dcol, int stride, int64_t d, const int *count, int64_t n,
                              cudaStream_t s) {
    init_state_kernel<<<elementwise_grid(d), 256, 0, s>>>(state, dcol, stride, d, count, n);
    return cudaGetLastError();
}

template <typename T, bool kDense>
static void smooth_t(const EvalParams &p, int64_t nnz, double c_loss, int grid, double *partial, cudaStream_t s) {
    row_smoothness_kernel<T, kDense><<<grid, kEvalBlock, 0, s>>>(p, nnz, c_loss, partial);
}

cudaError_t launch_max_row_smoothness(const EvalParams &p, int64_t nnz, int vtype, bool dense, double c_loss, int grid,
                                      double *partial, double *out, cudaStream_t s) {
    switch (vtype) {
    case kF32: dense ? smooth_t<float, true>(p, nnz, c_loss, grid, partial, s) : smooth_t<float, false>(p, nnz, c_loss, grid, partial, s); break;
    case kBF16: dense ? smooth_t<__nv_bfloat16, true>(p, nnz, c_loss, grid, partial, s) : smooth_t<__nv_bfloat16, false>(p, nnz, c_loss, grid, partial, s); break;
    case kF16: dense ? smooth_t<__half, true>(p, nnz, c_loss, grid, partial, s) : smooth_t<__half, false>(p, nnz, c_loss, grid, partial, s); break;
    default: return cudaErrorInvalidValue;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_reduce_partials(partial, grid, 1, out, s);
}

template <typename S>
static cudaError_t convert_from(const S *src, void *dst, int vtype, int64_t count, cudaStream_t s) {
    const int g = elementwise_grid(count);
    switch (vtype) {
    case kF32: convert_kernel<S, float><<<g, 256, 0, s>>>(src, (float *)dst, count); break;
    case kBF16: convert_kernel<S, __nv_bfloat16><<<g, 256, 0, s>>>(src, (__nv_bfloat16 *)dst, count); break;
    case kF16: convert_kernel<S, __half><<<g, 256, 0, s>>>(src, (__half *)dst, count); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_convert(const void *src, int src_dtype, void *dst, int vtype, int64_t count, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    switch (src_dtype) {
    case 0: return convert_from((const double *)src, dst, vtype, count, s);
    case 1: return convert_from((const float *)src, dst, vtype, count, s);
    case 2: return convert_from((const __nv_bfloat16 *)src, dst, vtype, count, s);
    case 3: return convert_from((const __half *)src, dst, vtype, count, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_labels(const double *lab64, float *lab32, int64_t n, cudaStream_t s) {
    labels_kernel<<<elementwise_grid(n), 256, 0, s>>>(lab64, lab32, n);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ compact layouts

// flag[0] |= 1 when a row holds two different stored values.
template <typename T>
__global__ void row_constant_kernel(const int64_t *row_ptr, const T *vals, int64_t n, int *flag) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = row_ptr[i], b = row_ptr[i + 1];
        if (b <= a) continue;
        const float v0 = to_f32(vals[a]);
        for (int64_t k = a + 1; k < b; ++k)
            if (to_f32(vals[k]) != v0) {
                atomicOr(flag, 1);
                break;
            }
    }
}

template <typename T>
__global__ void row_scale_kernel(const int64_t *row_ptr, const T *vals, int64_t n, float *scale) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        scale[i] = row_ptr[i + 1] > row_ptr[i] ? to_f32(vals[row_ptr[i]]) : 0.f;
}

__global__ void cols_to_u16_kernel(const int32_t *col, uint16_t *col16, int64_t nnz) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz; k += (int64_t)gridDim.x * blockDim.x)
        col16[k] = (uint16_t)col[k];
}

cudaError_t launch_row_constant_check(const int64_t *row_ptr, const void *values, int vtype, int64_t n, int *flag,
                                      cudaStream_t s) {
    const int g = elementwise_grid(n);
    switch (vtype) {
    case kF32: row_constant_kernel<float><<<g, 256, 0, s>>>(row_ptr, (const float *)values, n, flag); break;
    case kBF16: row_constant_kernel<__nv_bfloat16><<<g, 256, 0, s>>>(row_ptr, (const __nv_bfloat16 *)values, n, flag); break;
    case kF16: row_constant_kernel<__half><<<g, 256, 0, s>>>(row_ptr, (const __half *)values, n, flag); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_row_scale(const int64_t *row_ptr, const void *values, int vtype, int64_t n, float *scale,
                             cudaStream_t s) {
    const int g = elementwise_grid(n);
    switch (vtype) {
    case kF32: row_scale_kernel<float><<<g, 256, 0, s>>>(row_ptr, (const float *)values, n, scale); break;
    case kBF16: row_scale_kernel<__nv_bfloat16><<<g, 256, 0, s>>>(row_ptr, (const __nv_bfloat16 *)values, n, scale); break;
    case kF16: row_scale_kernel<__half><<<g, 256, 0, s>>>(row_ptr, (const __half *)values, n, scale); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_cols_to_u16(const int32_t *col, uint16_t *col16, int64_t nnz, cudaStream_t s) {
    if (nnz > 0) cols_to_u16_kernel<<<elementwise_grid(nnz), 256, 0, s>>>(col, col16, nnz);
    return cudaGetLastError();
}

}  // namespace asaga
