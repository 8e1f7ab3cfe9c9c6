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
// Latency: a row's CSR data does not depend on the solver state, so each
// warp stages it in shared memory ahead of time with asynchronous copies
// (cp.async, one commit group per update): the row_ptr entries and label of
// the row four updates ahead and the column indices and values of the row
// two updates ahead are requested just before the current row is processed,
// outside the window between its state reads and writes.
// Commit groups complete in order, so waiting for all but the newest group
// makes exactly the rows needed next available.  The window between reading
// x^ and writing x, which sets the overlap tau, is then one L2 gather, a
// warp reduction and the reductions back to L2.
//
// Layout: A in CSR (int64 row_ptr, int32 col_idx, values in fp32/bf16/fp16)
// or dense row-major; per-column state float4 {x, abar, D, 0}, so one
// 16-byte L2 read serves x^_v, abar_v and D_v and one 8-byte vector
// reduction updates x_v and abar_v.  Up to kRowCap entries of a row are
// staged (lane l owns entries l, l+32, ...); longer rows read the rest
// from global memory.
#include <algorithm>

#include "asaga_internal.h"
#include "device_common.cuh"

namespace asaga {

constexpr int kSlots = 4;
constexpr int kRowCap = 32 * kSlots;  // entries of a row staged in shared memory
// Entries kRowCap .. kRowCap + 32 kTailSlots - 1 of a long row are loaded
// from global memory into registers before the update's reads start, so that
// the read-to-write window holds only their state gathers; entries beyond
// are read inside the window (rare: rows of more than 256 entries).
constexpr int kTailSlots = 4;
constexpr int kStages = 4;            // staged CSR slices per warp (ring)
constexpr int kMetaRing = 8;          // staged row_ptr / label entries per warp (ring)

// Per-warp staging area in shared memory (4.3 KB).
struct __align__(16) WarpRing {
    int64_t start[kMetaRing];  // row_ptr[i]
    int64_t end[kMetaRing];    // row_ptr[i + 1]
    int64_t row[kMetaRing];    // i, or -1 past the end
    float label[kMetaRing];
    float scale[kMetaRing];    // the row's value (RowScale layout)
    int32_t col[kStages][kRowCap];  // int32 indices, or pairs of uint16 indices as aligned 32-bit words
    uint32_t val[kStages][kRowCap];  // raw 32-bit words: one fp32 or two 16-bit values
};

__device__ __forceinline__ void red_add_f32(float *p, float v) {
    asm volatile("red.relaxed.gpu.global.add.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
}

__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all_but_newest() {
    asm volatile("cp.async.wait_group 1;" ::: "memory");
}
// Commits every copy this thread has issued and waits for all of them.
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

template <typename T> __device__ __forceinline__ float staged_value(const uint32_t *words, int64_t start, int k);
template <> __device__ __forceinline__ float staged_value<float>(const uint32_t *words, int64_t, int k) {
    return __uint_as_float(words[k]);
}
template <> __device__ __forceinline__ float staged_value<__nv_bfloat16>(const uint32_t *words, int64_t start, int k) {
    const unsigned short h = reinterpret_cast<const unsigned short *>(words)[(int)(start & 1) + k];
    return __uint_as_float((unsigned)h << 16);
}
template <> __device__ __forceinline__ float staged_value<__half>(const uint32_t *words, int64_t start, int k) {
    const unsigned short h = reinterpret_cast<const unsigned short *>(words)[(int)(start & 1) + k];
    return __half2float(__ushort_as_half(h));
}

// Column of staged entry k: int32 words, or uint16 halves of aligned 32-bit
// words starting at the word that holds entry `start`.
template <typename I> __device__ __forceinline__ int staged_col(const int32_t *words, int64_t start, int k);
template <> __device__ __forceinline__ int staged_col<int32_t>(const int32_t *words, int64_t, int k) {
    return words[k];
}
template <> __device__ __forceinline__ int staged_col<uint16_t>(const int32_t *words, int64_t start, int k) {
    return reinterpret_cast<const uint16_t *>(words)[(int)(start & 1) + k];
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
    return sampled_row(P.sampling, P.seed, P.t_begin + (uint64_t)t, P.n);
}

// Lane 0 requests row i's row_ptr entries and label into meta slot m.
template <typename T, bool kDense>
__device__ __forceinline__ void stage_meta(const UpdateParams &P, WarpRing &R, int m, int64_t i, int lane) {
    if (lane != 0) return;
    R.row[m] = i;
    if (i < 0) return;
    if (kDense) {
        R.start[m] = i * P.d;
        R.end[m] = i * P.d + P.d;
    } else {
        cp_async8(&R.start[m], P.row_ptr + i);
        cp_async8(&R.end[m], P.row_ptr + i + 1);
    }
    cp_async4(&R.label[m], P.labels + i);
    if constexpr (IsRowScale<T>::value) cp_async4(&R.scale[m], static_cast<const float *>(P.values) + i);
}

// All lanes request the first kRowCap column indices and values of the row in
// meta slot m into stage st (16-bit values and indices travel as aligned
// 32-bit words; a RowScale row has no values to stage).
template <typename T, typename I, bool kDense>
__device__ __forceinline__ void stage_slice(const UpdateParams &P, WarpRing &R, int m, int st, int lane) {
    if (R.row[m] < 0) return;
    const int64_t start = R.start[m];
    const int64_t end = R.end[m];
    if (start < 0 || end < start || end > P.nnz) {  // a malformed row range: record it, copy nothing
        if (lane == 0) atomicOr(P.status, 4);
        return;
    }
    const int len = (int)(end - start);
    const int cnt = len < kRowCap ? len : kRowCap;
    if (!kDense) {
        const uint32_t *w = static_cast<const uint32_t *>(P.col_idx);
        if (sizeof(I) == 4) {
            for (int j = lane; j < cnt; j += 32) cp_async4(&R.col[st][j], w + start + j);
        } else {
            const int64_t w0 = start >> 1;
            const int nw = (int)(((start + cnt + 1) >> 1) - w0);
            for (int j = lane; j < nw; j += 32) cp_async4(&R.col[st][j], w + w0 + j);
        }
    }
    if constexpr (IsRowScale<T>::value) {
        return;
    } else if (sizeof(T) == 4) {
        const uint32_t *w = static_cast<const uint32_t *>(P.values);
        for (int j = lane; j < cnt; j += 32) cp_async4(&R.val[st][j], w + start + j);
    } else {
        const uint32_t *w = static_cast<const uint32_t *>(P.values);
        const int64_t w0 = start >> 1;
        const int nw = (int)(((start + cnt + 1) >> 1) - w0);
        for (int j = lane; j < nw; j += 32) cp_async4(&R.val[st][j], w + w0 + j);
    }
}

// The state-dependent part of one update: the inconsistent reads
// (begin_update), then the dot product, loss derivative and atomic adds
// (finish_update).
// kN register slots of 32 entries: the staged part (kSlots), plus for the
// single-problem sparse kernel the early-loaded tail of a long row (dense
// rows, and the batch's short rows, need none).
template <int kN> struct Update {
    int64_t i, start;
    int len;
    float label, alpha_hat, scale;
    int c[kN];
    float a[kN];
    float4 s[kN];
};

// The row's data (not the solver state): the staged part from shared memory,
// the next 32 kTailSlots entries of a long row from global memory.  Runs
// before the update's reads, outside the window that sets the overlap.
template <typename T, typename I, bool kDense, int kN>
__device__ __forceinline__ bool load_row(const UpdateParams &P, const WarpRing &R, int m, int st, int lane,
                                         Update<kN> &u) {
    u.i = R.row[m];
    u.start = R.start[m];
    const int64_t end = R.end[m];
    if (u.start < 0 || end < u.start || end > P.nnz) return false;  // recorded when it was staged
    u.len = (int)(end - u.start);
    u.label = R.label[m];
    u.scale = IsRowScale<T>::value ? R.scale[m] : 0.f;
#pragma unroll
    for (int q = 0; q < kN; ++q) {
        const int k = lane + 32 * q;
        u.c[q] = 0;
        u.a[q] = 0.f;
        if (k < u.len) {
            if (q < kSlots) {
                u.c[q] = kDense ? k : staged_col<I>(R.col[st], u.start, k);
                if constexpr (IsRowScale<T>::value)
                    u.a[q] = u.scale;
                else
                    u.a[q] = staged_value<T>(R.val[st], u.start, k);
            } else {
                u.c[q] = kDense ? k : col_stream<I>(P.col_idx, u.start + k);
                if constexpr (IsRowScale<T>::value)
                    u.a[q] = u.scale;
                else
                    u.a[q] = to_f32(ld_stream(static_cast<const T *>(P.values) + u.start + k));
            }
        }
    }
    return true;
}

// Issues the inconsistent reads of x^, abar, D (one 16-byte gather per
// entry) and alpha^_i: the start of the update's window.
template <int kN>
__device__ __forceinline__ void begin_update(const UpdateParams &P, int lane, Update<kN> &u) {
#pragma unroll
    for (int q = 0; q < kN; ++q) {
        u.s[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (lane + 32 * q < u.len) u.s[q] = ld_state(P.state + u.c[q] * (int64_t)P.stride);
    }
    u.alpha_hat = __ldcg(P.alpha + u.i);
}

// Dot product, loss derivative and the atomic adds to x, abar and alpha_i.
// Column and value of an entry past the register slots (global memory).
template <typename T, typename I, bool kDense, int kN>
__device__ __forceinline__ void tail_entry(const UpdateParams &P, const Update<kN> &u, int k, int &col,
                                          float &a) {
    col = kDense ? k : col_stream<I>(P.col_idx, u.start + k);
    if constexpr (IsRowScale<T>::value)
        a = u.scale;
    else
        a = to_f32(ld_stream(static_cast<const T *>(P.values) + u.start + k));
}

template <typename T, typename I, bool kDense, int kN>
__device__ __forceinline__ void finish_update(const UpdateParams &P, const Update<kN> &u, int lane) {
    const float4 *__restrict__ state = P.state;
    const int64_t stride = P.stride;
    float z = 0.f;
#pragma unroll
    for (int q = 0; q < kN; ++q) z = fmaf(u.a[q], u.s[q].x, z);
    for (int k = lane + 32 * kN; k < u.len; k += 32) {  // rest of a very long row
        int cc;
        float av;
        tail_entry<T, I, kDense, kN>(P, u, k, cc, av);
        z = fmaf(av, ld_state(state + cc * stride).x, z);
    }
    z = warp_sum(z);
    const float delta = phi_prime_f32(P.loss, z, u.label) - u.alpha_hat;  // same value in every lane

    const float gamma = P.gamma, lambda = P.lambda, inv_n = P.inv_n;
    if (P.plain_writes) {  // non-thread-safe x_v = x_v + dx (App. G.2 comparison): concurrent adds can be lost
#pragma unroll
        for (int q = 0; q < kN; ++q) {
            if (lane + 32 * q < u.len) {
                const float dx = -gamma * fmaf(delta, u.a[q], u.s[q].z * fmaf(lambda, u.s[q].x, u.s[q].y));
                float4 *ptr = P.state + u.c[q] * stride;
                const float4 cur = ld_state(ptr);
                __stcg(reinterpret_cast<float2 *>(ptr), make_float2(cur.x + dx, cur.y + delta * u.a[q] * inv_n));
            }
        }
        if (lane == 0) __stcg(P.alpha + u.i, __ldcg(P.alpha + u.i) + delta);
        return;
    }
#pragma unroll
    for (int q = 0; q < kN; ++q) {
        if (lane + 32 * q < u.len) {
            const float dx = -gamma * fmaf(delta, u.a[q], u.s[q].z * fmaf(lambda, u.s[q].x, u.s[q].y));
            red_add_v2(P.state + u.c[q] * stride, dx, delta * u.a[q] * inv_n);
        }
    }
    for (int k = lane + 32 * kN; k < u.len; k += 32) {
        int cc;
        float av;
        tail_entry<T, I, kDense, kN>(P, u, k, cc, av);
        const float4 sv = ld_state(state + cc * stride);
        const float dx = -gamma * fmaf(delta, av, sv.z * fmaf(lambda, sv.x, sv.y));
        red_add_v2(P.state + cc * stride, dx, delta * av * inv_n);
    }
    if (lane == 0) red_add_f32(P.alpha + u.i, delta);
}

// One warp's share of a launch: updates warp, warp + W, warp + 2W, ... of P.
// Iteration k processes the row of update warp + k W; before it, all commit
// groups but the newest are complete, which covers that row's staged slice
// and the row_ptr entries of row k + 2, whose slice is requested next.
template <typename T, typename I, bool kDense, int kN>
__device__ __forceinline__ void warp_updates(const UpdateParams &P, WarpRing &R, int warp, int lane) {
    const int64_t W = P.nwarps;
    uint64_t deadline = 0;
    if (P.deadline_ns) {  // budget relative to this warp's start (warp-uniform)
        const uint64_t now = __shfl_sync(kFull, globaltimer_ns(), 0);
        deadline = now + P.deadline_ns;
    }
    bool bad = false;
    // prologue: row_ptr entries of rows 0..3, then the slices of rows 0 and 1
    for (int k = 0; k < 4; ++k) stage_meta<T, kDense>(P, R, k, row_of(P, warp + k * W, bad), lane);
    cp_async_wait_all();
    __syncwarp();
    stage_slice<T, I, kDense>(P, R, 0, 0, lane);
    cp_async_commit();
    stage_slice<T, I, kDense>(P, R, 1, 1, lane);
    cp_async_commit();
    int64_t done = 0;
    for (int64_t k = 0;; ++k) {
        cp_async_wait_all_but_newest();
        __syncwarp();
        const int m = (int)(k & (kMetaRing - 1));
        if (R.row[m] < 0) break;
        // stage the slice of row k + 2 and the row_ptr entries of row k + 4 before
        // touching the state: the window between this update's reads and
        // writes (which sets the overlap tau) then holds no staging work
        const int m2 = (int)((k + 2) & (kMetaRing - 1));
        stage_slice<T, I, kDense>(P, R, m2, (int)((k + 2) & (kStages - 1)), lane);
        const bool more = R.row[(k + 3) & (kMetaRing - 1)] >= 0;
        stage_meta<T, kDense>(P, R, (int)((k + 4) & (kMetaRing - 1)), more ? row_of(P, warp + (k + 4) * W, bad) : -1,
                           lane);
        cp_async_commit();
        Update<kN> u;
        const bool ok = load_row<T, I, kDense, kN>(P, R, m, (int)(k & (kStages - 1)), lane, u);
        uint64_t t_read = 0;
        if (P.trace) t_read = globaltimer_ns();
        if (ok) {
            begin_update<kN>(P, lane, u);
            finish_update<T, I, kDense, kN>(P, u, lane);
        }
        if (P.trace && lane == 0) {
            P.trace[2 * (warp + k * W)] = t_read;
            P.trace[2 * (warp + k * W) + 1] = globaltimer_ns();
        }
        if (P.fence_each) {
            __threadfence();
            __syncwarp();
        }
        if ((deadline || P.cancel) && ((++done & 31) == 0)) {
            // the deadline every 32 updates; the host's cancel flag (a read of
            // mapped host memory) every 256
            int stop = 0;
            if (lane == 0) {
                if (deadline && globaltimer_ns() > deadline)
                    stop = 1;
                else if (P.cancel && (done & 255) == 0 && *P.cancel)
                    stop = 8;
            }
            stop = __shfl_sync(kFull, stop, 0);
            if (stop) {
                if (lane == 0) atomicOr(P.status, stop);
                break;
            }
        }
    }
    cp_async_wait_all();  // no copy may outlive the warp's staging area
    if (bad && lane == 0) atomicOr(P.status, 2);
}

template <typename T, typename I, bool kDense>
__global__ void __launch_bounds__(kUpdateBlock) update_kernel(const UpdateParams P) {
    __shared__ WarpRing rings[kUpdateBlock / 32];
    const int lane = threadIdx.x & 31;
    const int warp = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
    if (warp >= P.nwarps) return;
    warp_updates<T, I, kDense, kDense ? kSlots : kSlots + kTailSlots>(P, rings[threadIdx.x >> 5], warp, lane);
}

// Many independent problems in one launch: block b serves instance
// inst = the last i with block_begin[i] <= b, whose parameters are copied to
// shared memory once; its warps split that instance's updates.
template <typename T, typename I, bool kDense>
__global__ void __launch_bounds__(kBatchBlock) batch_update_kernel(const UpdateParams *__restrict__ params,
                                                                   const int *__restrict__ block_begin, int count) {
    __shared__ UpdateParams sp;
    __shared__ int s_inst;
    __shared__ WarpRing rings[kBatchBlock / 32];
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
    warp_updates<T, I, kDense, kSlots>(sp, rings[threadIdx.x >> 5], warp, lane);
}

struct UpdateLaunch {
    const UpdateParams &p;
    int grid, block;
    cudaStream_t s;
    template <typename T, typename I, bool kDense> cudaError_t run() const {
        update_kernel<T, I, kDense><<<grid, block, 0, s>>>(p);
        return cudaGetLastError();
    }
};

cudaError_t launch_update(const UpdateParams &p, int layout, bool dense, int grid, int block, cudaStream_t s) {
    return with_layout(layout, dense, UpdateLaunch{p, grid, block, s}, cudaErrorInvalidValue);
}

struct BatchUpdateLaunch {
    const UpdateParams *params;
    const int *block_begin;
    int count, grid;
    cudaStream_t s;
    template <typename T, typename I, bool kDense> cudaError_t run() const {
        batch_update_kernel<T, I, kDense><<<grid, kBatchBlock, 0, s>>>(params, block_begin, count);
        return cudaGetLastError();
    }
};

cudaError_t launch_batch_update(const UpdateParams *params, const int *block_begin, int count, int grid, int layout,
                                bool dense, cudaStream_t s) {
    return with_layout(layout, dense, BatchUpdateLaunch{params, block_begin, count, grid, s}, cudaErrorInvalidValue);
}

// Resident blocks per SM of the update kernels (from the occupancy calculator).
struct UpdateOccupancy {
    bool batch;
    template <typename T, typename I, bool kDense> int run() const {
        int nb = 0;
        const cudaError_t e =
            batch ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_update_kernel<T, I, kDense>, kBatchBlock, 0)
                  : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, update_kernel<T, I, kDense>, kUpdateBlock, 0);
        return e == cudaSuccess && nb > 0 ? nb : 1;
    }
};

int batch_update_max_blocks_per_sm(int layout, bool dense) { return with_layout(layout, dense, UpdateOccupancy{true}, 1); }

int update_max_blocks_per_sm(int layout, bool dense) { return with_layout(layout, dense, UpdateOccupancy{false}, 1); }

__global__ void sample_rows_kernel(uint64_t seed, int64_t n, int sampling, uint64_t t_begin, int64_t count,
                                   int64_t *rows) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < count; j += (int64_t)gridDim.x * blockDim.x)
        rows[j] = sampled_row(sampling, seed, t_begin + (uint64_t)j, n);
}

cudaError_t launch_sample_rows(uint64_t seed, int64_t n, int sampling, uint64_t t_begin, int64_t count,
                               int64_t *rows, cudaStream_t stream) {
    if (count <= 0) return cudaSuccess;
    const int grid = (int)std::min<int64_t>(4096, (count + 255) / 256);
    sample_rows_kernel<<<grid, 256, 0, stream>>>(seed, n, sampling, t_begin, count, rows);
    return cudaGetLastError();
}

}  // namespace asaga
