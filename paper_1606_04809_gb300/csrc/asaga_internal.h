// Internal declarations shared by the solver's CUDA translation units:
// launch parameters of every kernel and the host-side launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

namespace asaga {

// Device element type of A's values; kRowScale: one float32 value per row
// (every stored value of the row is equal, e.g. binary rows scaled to unit
// norm), held in the `values` array of n entries.
enum ValType : int { kF32 = 1, kBF16 = 2, kF16 = 3, kRowScale = 4 };
// A layout, as the steady-state kernels see A: a ValType, or'ed with
// kIdx16 when the column indices are stored as uint16 (d <= 65536).
constexpr int kIdx16 = 8;

// Per-column solver state: the mutable pair float2 {x_v, abar_v} (8 bytes,
// gathered by one load and updated by one 2-wide vector reduction), columns
// spaced `stride` float2s apart; and the constant reweighting D_v in an
// array of its own, read through the non-coherent (L1-cached) path, so that
// the lines the updates contend for hold only mutable state.


// Launch parameters of the asynchronous update kernel (one update = one
// sampled row, Algorithm 2).
//
// Cores.  Each concurrent update runs on one "core": a single warp, or, on
// the multi-warp row path, a group of `group` warps of one block that split
// the row's entries, add their partial dot products through shared memory
// and apply the same delta.  Rows longer than `threshold` entries take the
// multi-warp path (threshold 0: every row; < 0: none).  Blocks
// [0, short_blocks) hold `wpb` single-warp cores each and the others
// wpb / group multi-warp cores; core j of a path takes the updates
// t = j, j + cores, j + 2 cores, ... of the launch whose rows belong to that
// path (long_bits tells a row's path when both paths are in use), so every
// update is applied exactly once whatever the split.
struct UpdateParams {
    int64_t n, d;
    int64_t nnz;              // entries of A (n*d for dense); staged row ranges are checked against it
    const int64_t *row_ptr;   // n+1 (sparse) or nullptr (dense)
    const void *col_idx;      // nnz int32 or uint16 (by layout), or nullptr (dense)
    const void *values;       // nnz (or n*d) of the storage type, or n row values (kRowScale)
    const float *labels;      // n, float32 copy for the update
    float *alpha;             // n, scalar memory per sample
    float2 *state;            // d * stride: {x_v, abar_v}
    const float *dcol;        // d: D_v
    int stride;               // float2s between consecutive columns
    int loss;                 // 0 logistic, 1 squared
    float gamma, lambda, inv_n;
    uint64_t seed;            // sampler seed
    int sampling;             // 0 uniform with replacement, 1 one permutation per epoch
    uint64_t t_begin;         // global index of this launch's first update
    int64_t count;            // updates in this launch
    int short_cores;          // single-warp cores
    int long_cores;           // multi-warp cores (group warps each)
    int group;                // warps per multi-warp core: 1, 2, 4 or 8
    int64_t threshold;        // rows longer than this take the multi-warp path (0: all, < 0: none)
    int wpb;                  // warps per block (a multiple of group)
    int short_blocks;         // blocks of single-warp cores (the first ones)
    const uint32_t *long_bits;  // bit i set: row i takes the multi-warp path; nullptr when one path takes all rows
    float *tail_c;            // per core tail_stride floats: the update's term D_v (abar_v + lambda x^_v) for
    int64_t tail_stride;      //   entries past the register slots (nullptr / 0 when no row has such entries)
    const int64_t *idx;       // explicit row sequence (deterministic replay) or nullptr
    int fence_each;           // 1: fence after every update (single-core order)
    int plain_writes;         // 1: non-atomic load-add-store instead of reductions (diagnostic)
    int draw_ahead;           // 1: the next row is drawn while the update's gathers are in flight
    uint64_t deadline_ns;     // %globaltimer deadline, 0 = none
    const volatile int *cancel;  // nonzero: stop (a flag in mapped host memory), or nullptr
    int *status;              // bit 0: timed out, bit 1: bad index, bit 2: malformed row range, bit 3: cancelled,
                              // bit 4: a staging copy did not complete in time, bit 5: tail scratch too small
    uint64_t *trace;          // 2 * count: %globaltimer before the reads / after the writes of update t (or nullptr)
};

// Float64 evaluation parameters (objective, gradient, abar recomputation).
struct EvalParams {
    int64_t n, d;
    const int64_t *row_ptr;
    const void *col_idx;      // int32 or uint16 by layout (int32 in the set-up kernels)
    const void *values;       // per entry, or per row (kRowScale)
    const double *labels;     // n, float64
    const float *alpha;       // n
    float2 *state;            // {x_v, abar_v}, stride float2s apart
    const float *dcol;        // D_v
    int stride;
    int loss;
    double lambda;
    const int *hot_slot;      // d entries: shared-memory slot of a frequent column, -1 otherwise (may be nullptr)
    const int *hot_col;       // n_hot entries: column of each slot
    int n_hot;
    double *acc;              // d float64 accumulators (the batched abar recomputation)
};

constexpr int kUpdateBlock = 256;  // threads per block of the update kernel
constexpr int kBatchBlock = 128;   // threads per block of the batched update kernel (4 warps)
constexpr int kMaxGroup = 8;       // warps of the widest multi-warp core
constexpr int kEvalBlock = 256;
constexpr int kMaxPartials = 4096; // max blocks of the float64 row kernels
constexpr int kMaxHot = 2048;      // frequent columns accumulated per block in shared memory

// api.cu: the text asaga_last_error(NULL) returns on this host thread.
void set_thread_error(const std::string &msg);

// update.cu
// rows[j] = the row of update t_begin + j (device buffer of count entries)
cudaError_t launch_sample_rows(uint64_t seed, int64_t n, int sampling, uint64_t t_begin, int64_t count,
                               int64_t *rows, cudaStream_t stream);
// grid = short_blocks + blocks of multi-warp cores, p.wpb warps per block.
cudaError_t launch_update(const UpdateParams &p, int layout, bool dense, int grid, cudaStream_t s);
// dynamic shared memory of an update block of wpb warps
size_t update_smem_bytes(int wpb);
int update_max_blocks_per_sm(int layout, bool dense);
// register slots of 32 entries per lane of the update kernels: a core of g
// warps keeps 32 g update_register_slots(...) entries of a row in registers
int update_register_slots(bool dense, bool batch);
// bits[i / 32] bit i % 32 <- (row_ptr[i+1] - row_ptr[i] > threshold); sums[0] += entries of
// such rows, sums[1] += their number (sums: 2 int64, zeroed by the caller)
cudaError_t launch_row_classes(const int64_t *row_ptr, int64_t n, int64_t threshold, uint32_t *bits,
                               unsigned long long *sums, cudaStream_t s);
// params[count] and block_begin[count] in device memory; instance i owns blocks
// [block_begin[i], block_begin[i+1]) (the last one up to grid).
cudaError_t launch_batch_update(const UpdateParams *params, const int *block_begin, int count, int grid, int layout,
                                bool dense, cudaStream_t s);
int batch_update_max_blocks_per_sm(int layout, bool dense);

// eval.cu
// partial[0..grid) <- per-block sums of phi_i(a_i.x); partial[grid..2grid) <- sums of x_v^2.
cudaError_t launch_objective_rows(const EvalParams &p, int layout, bool dense, int grid,
                                  double *partial, cudaStream_t s);
// out[0] <- (sum partial[0..grid))/n + lambda/2 (sum partial[grid..2grid)).
cudaError_t launch_objective_finish(const double *partial, int grid, double inv_n, double lambda,
                                    double *out, cudaStream_t s);
// Objectives of `count` instances in one launch of grid x count blocks:
// partial holds 2 * grid * count doubles; f_out[i] receives instance i's f.
cudaError_t launch_batch_objective(const EvalParams *params, int count, int grid, int layout, bool dense,
                                   double *partial, double *f_out, cudaStream_t s);
// acc[v] += sum_i w_i a_iv with w_i = phi'_i(a_i.x)/n (mode 0) or alpha_i/n (mode 1).
cudaError_t launch_scatter_rows(const EvalParams &p, int layout, bool dense, int mode, int grid,
                                double *acc, cudaStream_t s);
// mode 0 (gradient): acc[v] += lambda x_v; partial[b] <- block sums of acc[v]^2.
// mode 1 (abar):     partial[b] <- block max |abar_v - acc[v]|, then abar_v <- (float)acc[v].
cudaError_t launch_column_finish(const EvalParams &p, int mode, int grid, double *acc,
                                 double *partial, cudaStream_t s);
// out[0] <- sum (mode 0) or max (mode 1) of partial[0..grid).
cudaError_t launch_reduce_partials(const double *partial, int grid, int mode, double *out,
                                   cudaStream_t s);

// The abar recomputation of `count` instances in three launches:
// acc_i <- 0, acc_i[v] += sum_r (alpha_r / n_i) a_rv (a warp per row, grid x
// count blocks), then abar_v <- (float)acc_v and drift_out[i] <- max_v
// |abar_v(before) - acc_v|.  An instance with n = d = 0 is skipped.
// partial holds grid * count doubles.
cudaError_t launch_batch_recompute(const EvalParams *params, int count, int grid, int layout, bool dense,
                                   int max_hot, double *partial, double *drift_out, cudaStream_t s);

// prep (eval.cu).  These run while the host is still checking the problem,
// so they skip columns outside [0, d) and row ranges outside [0, nnz].
cudaError_t launch_count_columns(const int32_t *col_idx, int64_t nnz, int64_t d, int *count, cudaStream_t s);
// state[v] <- {0, 0}, dcol[v] <- D_v = n/count_v (0 if count_v = 0); count may be nullptr (dense: D = 1).
cudaError_t launch_init_state(float2 *state, float *dcol, int stride, int64_t d, const int *count, int64_t n,
                              cudaStream_t s);
// out[0] <- max_i (c |a_i|^2 + lambda max_{v in S_i} D_v) (float64) over the stored
// values; needs D in dcol.  Set-up layout: int32 columns, one value per entry.
cudaError_t launch_max_row_smoothness(const EvalParams &p, int64_t nnz, int vtype, bool dense, double c_loss, int grid,
                                      double *partial, double *out, cudaStream_t s);
// dst (vtype) <- src (src_dtype: 0 f64, 1 f32, 2 bf16, 3 f16), count elements.
cudaError_t launch_convert(const void *src, int src_dtype, void *dst, int vtype, int64_t count,
                           cudaStream_t s);
cudaError_t launch_labels(const double *lab64, float *lab32, int64_t n, cudaStream_t s);
// Compact layouts (set-up): flag[0] |= 1 if some row holds two different
// stored values (vtype, per-entry values); scale[i] <- the value of row i
// (0 for an empty row); col16[k] <- col[k].
cudaError_t launch_row_constant_check(const int64_t *row_ptr, const void *values, int vtype, int64_t n, int *flag,
                                      cudaStream_t s);
cudaError_t launch_row_scale(const int64_t *row_ptr, const void *values, int vtype, int64_t n, float *scale,
                             cudaStream_t s);
cudaError_t launch_cols_to_u16(const int32_t *col, uint16_t *col16, int64_t nnz, cudaStream_t s);

}  // namespace asaga
