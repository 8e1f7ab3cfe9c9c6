// Host side of the C ABI declared in include/asaga.h: validation, device
// layout, set-up (D, L, gamma), the segment loop of asaga_run and the float64
// evaluations.  All device work of a context is ordered on one CUDA stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <system_error>
#include <thread>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "asaga.h"
#include "asaga_internal.h"
#include "tune_rules.h"

using namespace asaga;

struct asaga_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int sms = 1;

    int64_t n = 0, d = 0, nnz = 0, max_row_len = 0;
    bool dense = false;
    int loss = 0;
    int vtype = kF32;   // storage type of the values (set-up layout)
    int layout = kF32;  // layout the steady-state kernels read: vtype or kRowScale, | kIdx16
    double lambda = 0, gamma = 0, L = 0, delta = 0;
    int stride = 1;
    int warps = 1;
    int resident_warps = 1;
    double gamma_base = 0;  // options.gamma, or 1/(3L)
    bool deterministic = false;
    bool plain_writes = false;
    int sampling = 0;              // ASAGA_SAMPLE_UNIFORM or ASAGA_SAMPLE_PERMUTATION
    bool spread = false;           // update kernel: warps spread over the SMs (else 8 per block)
    // row paths: rows longer than row_threshold entries (0: all, < 0: none)
    // are updated by cores of row_group warps (the multi-warp row path)
    int row_group = 1;
    int64_t row_threshold = -1;
    // 1: the next row is drawn while an update's gathers are in flight
    int draw_ahead = 0;
    uint32_t *long_bits = nullptr;   // bit i: row i is longer than bits_threshold
    int64_t bits_threshold = -1;     // the threshold long_bits was built for (-1: not built)
    double long_share = 0;           // fraction of the nonzeros in rows longer than bits_threshold
    unsigned long long *d_sums = nullptr;
    float *tail_c = nullptr;         // per-core scratch for entries past the register slots
    int64_t tail_floats = 0;
    uint64_t seed = 0;
    int epochs_per_segment = 1;
    int abar_every = 0;
    double timeout_s = 0;
    int64_t updates_done = 0;
    int64_t segments_done = 0;  // over the context's life: the abar recomputation cadence
    int eval_grid = 1;
    int64_t launches = 0;
    int64_t device_bytes = 0;

    // device buffers
    int64_t *row_ptr = nullptr;
    int32_t *col_idx = nullptr;   // freed once compacted to col16
    uint16_t *col16 = nullptr;    // compact layout: uint16 column indices (d <= 65536)
    void *values = nullptr;       // freed once compacted to row_scale
    float *row_scale = nullptr;   // compact layout: one value per row
    float *lab32 = nullptr;
    double *lab64 = nullptr;
    float *alpha = nullptr;
    float2 *state = nullptr;      // {x_v, abar_v}, stride float2s apart
    float *dcol = nullptr;        // D_v
    double *acc64 = nullptr;
    double *partial = nullptr;
    double *dout = nullptr;  // [0] f, [1..] small results
    int *status = nullptr;
    int *hot_slot = nullptr;  // d: shared-memory slot of a frequent column or -1
    int *hot_col = nullptr;   // n_hot: column of each slot
    int n_hot = 0;
    int64_t *idx_buf = nullptr;
    int64_t idx_cap = 0;
    double *hout = nullptr;  // pinned mirror of dout
    int *hstatus = nullptr;  // pinned
    int *h_cancel = nullptr;  // mapped pinned flag set by asaga_cancel
    int *d_cancel = nullptr;  // its device address
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};

    std::string err;
};

// Many independent problems solved together (see asaga_batch_create).
struct asaga_batch {
    int count = 0;
    std::vector<asaga_ctx *> ctx;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0;
    int layout = kF32;  // the instances' common layout (ValType | kIdx16)
    int cancel = 0;     // set by asaga_batch_cancel (atomic)
    bool dense = false;
    int epochs_per_segment = 1;
    int abar_every = 0;
    int64_t segments_done = 0;  // over the batch's life: the abar recomputation cadence
    int resident_blocks = 1;
    std::vector<int> warps;        // per instance, a multiple of 4 (one block = 4 warps)
    std::vector<int> block_begin;  // first block of each instance
    int grid = 0;
    int eval_grid = 1;             // blocks per instance in the batched objective
    UpdateParams *d_up = nullptr, *h_up = nullptr;
    EvalParams *d_ev = nullptr, *h_ev = nullptr;  // h_ev pinned, uploaded every segment
    std::vector<EvalParams> ev_full;              // every instance's evaluation parameters
    int *d_block_begin = nullptr;
    double *d_partial = nullptr, *d_f = nullptr, *h_f = nullptr;
    double *d_rpartial = nullptr, *d_drift = nullptr, *h_drift = nullptr;  // the batched abar recomputation
    int recompute_grid = 1;
    int max_hot = 0;
    int *d_status = nullptr, *h_status = nullptr;  // the update kernel's status bits of every instance
    cudaGraphExec_t graph = nullptr;     // segment: update launch, objectives
    cudaGraphExec_t graph_rc = nullptr;  // the same with the abar recomputation after the updates
    cudaEvent_t ev[2] = {nullptr, nullptr};
    int64_t launches = 0;
    std::string err;
};

namespace {

thread_local std::string g_create_err;

const char *kStatusNames[] = {"ASAGA_OK",        "ASAGA_EINVAL",    "ASAGA_ENOMEM",        "ASAGA_ECUDA",
                              "ASAGA_ETIMEOUT",  "ASAGA_EDIVERGED", "ASAGA_ENOTCONVERGED", "ASAGA_ECANCELLED"};

// NVTX range for profilers (a no-op unless a tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

asaga_status fail(std::string *err, asaga_status s, const std::string &msg) {
    if (err) *err = msg;
    return s;
}

asaga_status cuda_fail(std::string *err, cudaError_t e, const char *what) {
    cudaGetLastError();  // clear a sticky-free error
    if (err) *err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? ASAGA_ENOMEM : ASAGA_ECUDA;
}

#define CK(call, what)                                                   \
    do {                                                                 \
        cudaError_t e_ = (call);                                         \
        if (e_ != cudaSuccess) return cuda_fail(err, e_, what);          \
    } while (0)

size_t dtype_size(int dt) {
    switch (dt) {
    case ASAGA_F64: return 8;
    case ASAGA_F32: return 4;
    case ASAGA_BF16:
    case ASAGA_F16: return 2;
    default: return 0;
    }
}

// First non-finite value among entries [a, b) of an array of dtype dt, or -1
// (one tight loop per type; the 16-bit types by their exponent bits).
int64_t first_nonfinite(const void *vals, int dt, int64_t a, int64_t b) {
    switch (dt) {
    case ASAGA_F64:
        for (int64_t k = a; k < b; ++k)
            if (!std::isfinite(((const double *)vals)[k])) return k;
        return -1;
    case ASAGA_F32:
        for (int64_t k = a; k < b; ++k)
            if (!std::isfinite(((const float *)vals)[k])) return k;
        return -1;
    case ASAGA_BF16:
        for (int64_t k = a; k < b; ++k)
            if ((((const uint16_t *)vals)[k] & 0x7F80u) == 0x7F80u) return k;
        return -1;
    case ASAGA_F16:
        for (int64_t k = a; k < b; ++k)
            if ((((const uint16_t *)vals)[k] & 0x7C00u) == 0x7C00u) return k;
        return -1;
    default: return a < b ? a : -1;
    }
}

// Repeated-column check of one row at a time: an open-addressing set of the
// row's columns whose slots carry the row's stamp, so stale slots of earlier
// rows count as empty and nothing is cleared between rows.  Sized to at
// least twice the row (so it stays in L1 for ordinary rows, whatever d is).
class RowColumnSet {
  public:
    // Starts a row of len entries.
    void begin(int64_t len) {
        size_t cap = 64;
        while ((int64_t)cap < 2 * len) cap <<= 1;
        if (slot_.size() < cap) slot_.assign(cap, 0);
        mask_ = (uint32_t)(cap - 1);
        if (++stamp_ == 0) {  // the stamp wrapped: every slot is stale by clearing
            std::fill(slot_.begin(), slot_.end(), 0);
            stamp_ = 1;
        }
    }
    // False if c is already in the row.
    bool insert(int32_t c) {
        const uint64_t tagged = ((uint64_t)stamp_ << 32) | (uint32_t)c;
        uint32_t h = ((uint32_t)c * 2654435761u) & mask_;
        while ((uint32_t)(slot_[h] >> 32) == stamp_) {
            if (slot_[h] == tagged) return false;
            h = (h + 1) & mask_;
        }
        slot_[h] = tagged;
        return true;
    }

  private:
    std::vector<uint64_t> slot_;
    uint32_t mask_ = 0;
    uint32_t stamp_ = 0;
};

template <typename T>
asaga_status dev_alloc(T **p, size_t count, asaga_ctx *c, std::string *err, const char *what) {
    size_t bytes = count * sizeof(T);
    if (bytes == 0) bytes = sizeof(T);
    cudaError_t e = cudaMalloc((void **)p, bytes);
    if (e != cudaSuccess) return cuda_fail(err, e, what);
    c->device_bytes += (int64_t)bytes;
    return ASAGA_OK;
}

#define TRY(expr)                                 \
    do {                                          \
        asaga_status s_ = (expr);                 \
        if (s_ != ASAGA_OK) return s_;            \
    } while (0)

std::mutex g_max_mutex;

// Runs body(lo, hi, &error) over contiguous chunks of [0, count) on up to
// max_threads host threads (at least min_chunk items each).  Returns false
// with the error of the lowest failing chunk.
template <class F>
bool parallel_check(int64_t count, int64_t min_chunk, int max_threads, F body, std::string *msg) {
    if (count <= 0) return true;
    const int64_t hw = std::max<int64_t>(1, (int64_t)std::thread::hardware_concurrency());
    const int nt = (int)std::max<int64_t>(1, std::min<int64_t>({count / std::max<int64_t>(1, min_chunk), hw,
                                                               (int64_t)max_threads}));
    std::vector<std::string> errs(nt);
    if (nt == 1) {
        body(0, count, &errs[0]);
    } else {
        std::vector<std::thread> th;
        th.reserve(nt);
        for (int t = 0; t < nt; ++t) {
            const int64_t lo = count * t / nt, hi = count * (t + 1) / nt;
            try {
                th.emplace_back([&, t, lo, hi] { body(lo, hi, &errs[t]); });
            } catch (const std::system_error &) {  // no more threads: this block on the caller's
                body(lo, hi, &errs[t]);
            }
        }
        for (auto &x : th) x.join();
    }
    for (auto &e : errs)
        if (!e.empty()) {
            *msg = e;
            return false;
        }
    return true;
}

// Checks of the problem and options that need no pass over the data.
asaga_status validate_args(const asaga_problem *p, const asaga_options *o, std::string *err) {
    if (!p || !o) return fail(err, ASAGA_EINVAL, "problem or options is NULL");
    if (p->n < 1 || p->d < 1) return fail(err, ASAGA_EINVAL, "n and d must be >= 1");
    if (p->d > (int64_t)INT32_MAX) return fail(err, ASAGA_EINVAL, "d must fit in int32");
    if (o->loss != ASAGA_LOSS_LOGISTIC && o->loss != ASAGA_LOSS_SQUARED)
        return fail(err, ASAGA_EINVAL, "unknown loss");
    if (!std::isfinite(o->lambda) || o->lambda < 0) return fail(err, ASAGA_EINVAL, "lambda must be finite and >= 0");
    if (!std::isfinite(o->gamma)) return fail(err, ASAGA_EINVAL, "gamma must be finite");
    if (o->storage_dtype != ASAGA_F32 && o->storage_dtype != ASAGA_BF16 && o->storage_dtype != ASAGA_F16)
        return fail(err, ASAGA_EINVAL, "storage_dtype must be F32, BF16 or F16");
    if (dtype_size(p->values_dtype) == 0) return fail(err, ASAGA_EINVAL, "unknown values_dtype");
    if (o->epochs_per_segment < 0 || o->abar_recompute_every < 0 || o->max_warps < 0 ||
        o->column_stride < 0 || !(o->timeout_s >= 0))
        return fail(err, ASAGA_EINVAL, "negative option");
    if (o->sampling != ASAGA_SAMPLE_UNIFORM && o->sampling != ASAGA_SAMPLE_PERMUTATION)
        return fail(err, ASAGA_EINVAL, "unknown sampling");
    if (o->sampling == ASAGA_SAMPLE_PERMUTATION && p->n > ((int64_t)1 << 62))
        return fail(err, ASAGA_EINVAL, "permutation sampling needs n <= 2^62");
    if (!p->values || !p->labels) return fail(err, ASAGA_EINVAL, "values or labels is NULL");
    if (p->dense) {
        if (p->d > 0 && p->n > INT64_MAX / p->d) return fail(err, ASAGA_EINVAL, "n*d overflows");
        if (p->nnz != 0 && p->nnz != p->n * p->d)
            return fail(err, ASAGA_EINVAL, "dense problem needs nnz = n*d (or 0)");
    } else {
        if (p->nnz < 0) return fail(err, ASAGA_EINVAL, "nnz < 0");
        if (!p->row_ptr || (!p->col_idx && p->nnz > 0)) return fail(err, ASAGA_EINVAL, "row_ptr or col_idx is NULL");
    }
    return ASAGA_OK;
}

// One pass over the rows on host threads (device inputs are copied to the
// host first): labels finite (and +-1 for logistic), row_ptr from 0 to nnz
// and non-decreasing, columns in [0, d) and not repeated within a row, values
// finite.  Threads take contiguous blocks of rows and the error reported is
// the one of the first bad row.  Fills max_row_len.  Call after
// validate_args.
asaga_status validate_content(const asaga_problem *p, const asaga_options *o, int64_t *max_row_len,
                              std::string *err) {
    const int64_t nnz = p->dense ? p->n * p->d : p->nnz;
    const size_t vsz = dtype_size(p->values_dtype);
    std::vector<int64_t> rp_h;
    std::vector<int32_t> ci_h;
    std::vector<double> lab_h;
    std::vector<unsigned char> val_h;
    const int64_t *rp = p->row_ptr;
    const int32_t *ci = p->col_idx;
    const double *lab = p->labels;
    const void *val = p->values;
    if (p->on_device) {
        cudaError_t e;
        lab_h.resize(p->n);
        val_h.resize((size_t)nnz * vsz);
        if ((e = cudaMemcpy(lab_h.data(), p->labels, p->n * sizeof(double), cudaMemcpyDeviceToHost)) != cudaSuccess)
            return cuda_fail(err, e, "copy labels for validation");
        if (nnz > 0 &&
            (e = cudaMemcpy(val_h.data(), p->values, (size_t)nnz * vsz, cudaMemcpyDeviceToHost)) != cudaSuccess)
            return cuda_fail(err, e, "copy values for validation");
        lab = lab_h.data();
        val = val_h.data();
        if (!p->dense) {
            rp_h.resize(p->n + 1);
            ci_h.resize(nnz);
            if ((e = cudaMemcpy(rp_h.data(), p->row_ptr, (p->n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost)) !=
                cudaSuccess)
                return cuda_fail(err, e, "copy row_ptr for validation");
            if (nnz > 0 &&
                (e = cudaMemcpy(ci_h.data(), p->col_idx, nnz * sizeof(int32_t), cudaMemcpyDeviceToHost)) != cudaSuccess)
                return cuda_fail(err, e, "copy col_idx for validation");
            rp = rp_h.data();
            ci = ci_h.data();
        }
    }
    if (!p->dense && (rp[0] != 0 || rp[p->n] != nnz))
        return fail(err, ASAGA_EINVAL, "row_ptr must start at 0 and end at nnz");
    const int loss = o->loss;
    const int vdt = p->values_dtype;
    const int64_t d = p->d;
    const bool dense = p->dense != 0;
    int64_t mrl = dense ? d : 0;
    std::string msg;
    // repeated columns: up to 2^18 columns each thread stamps a d-sized array
    // with the row (it stays in a core's L2); beyond, a per-row set
    const bool stamps = !dense && d <= (1 << 18);
    if (!parallel_check(p->n, 1 << 14, 32, [&](int64_t lo, int64_t hi, std::string *e) {
            RowColumnSet seen;
            std::vector<uint32_t> stamp(stamps ? d : 0, 0);
            int64_t m = 0;
            for (int64_t i = lo; i < hi; ++i) {
                if (!std::isfinite(lab[i])) return void(*e = "non-finite label at row " + std::to_string(i));
                if (loss == ASAGA_LOSS_LOGISTIC && lab[i] != 1.0 && lab[i] != -1.0)
                    return void(*e = "logistic label not +-1 at row " + std::to_string(i));
                int64_t a = i * d, b = (i + 1) * d;
                if (!dense) {
                    // a bad range is reported before anything in it is read
                    if (rp[i] < 0 || rp[i + 1] < rp[i])
                        return void(*e = "row_ptr decreases at row " + std::to_string(i));
                    if (rp[i + 1] > nnz) return void(*e = "row_ptr passes nnz at row " + std::to_string(i));
                    a = rp[i];
                    b = rp[i + 1];
                    const int64_t len = b - a;
                    if (len > INT32_MAX) return void(*e = "row too long");
                    m = len > m ? len : m;
                    // the usual case, columns in increasing order: no repeats, and the
                    // range follows from the first and last (checked without the
                    // random access of the general check, which other rows take)
                    bool sorted = len == 0 || (ci[a] >= 0 && ci[b - 1] < d);
                    for (int64_t k = a + 1; sorted && k < b; ++k) sorted = ci[k] > ci[k - 1];
                    if (sorted) {
                        // nothing more to check for the columns
                    } else if (stamps) {
                        const uint32_t tag = (uint32_t)(i - lo + 1);
                        for (int64_t k = a; k < b; ++k) {
                            const int32_t c = ci[k];
                            if (c < 0 || c >= d)
                                return void(*e = "column index out of range at entry " + std::to_string(k));
                            if (stamp[c] == tag) return void(*e = "repeated column in row " + std::to_string(i));
                            stamp[c] = tag;
                        }
                    } else {
                        seen.begin(len);
                        for (int64_t k = a; k < b; ++k) {
                            const int32_t c = ci[k];
                            if (c < 0 || c >= d)
                                return void(*e = "column index out of range at entry " + std::to_string(k));
                            if (!seen.insert(c)) return void(*e = "repeated column in row " + std::to_string(i));
                        }
                    }
                }
                const int64_t bad = first_nonfinite(val, vdt, a, b);
                if (bad >= 0) return void(*e = "non-finite value at entry " + std::to_string(bad));
            }
            std::lock_guard<std::mutex> g(g_max_mutex);
            mrl = m > mrl ? m : mrl;
        }, &msg))
        return fail(err, ASAGA_EINVAL, msg);
    *max_row_len = mrl;
    return ASAGA_OK;
}

// Column indices and values as the steady-state kernels read them.
const void *layout_cols(const asaga_ctx *c) {
    return (c->layout & kIdx16) ? (const void *)c->col16 : (const void *)c->col_idx;
}
const void *layout_values(const asaga_ctx *c) {
    return (c->layout & ~kIdx16) == kRowScale ? (const void *)c->row_scale : c->values;
}

EvalParams eval_params(const asaga_ctx *c) {
    EvalParams e;
    e.n = c->n;
    e.d = c->d;
    e.row_ptr = c->row_ptr;
    e.col_idx = layout_cols(c);
    e.values = layout_values(c);
    e.labels = c->lab64;
    e.alpha = c->alpha;
    e.state = c->state;
    e.dcol = c->dcol;
    e.stride = c->stride;
    e.loss = c->loss;
    e.lambda = c->lambda;
    e.hot_slot = c->hot_slot;
    e.hot_col = c->hot_col;
    e.n_hot = c->n_hot;
    e.acc = c->acc64;
    return e;
}

// Launches the float64 objective; result lands in c->dout[0].
asaga_status enqueue_objective(asaga_ctx *c, std::string *err) {
    const EvalParams e = eval_params(c);
    CK(launch_objective_rows(e, c->layout, c->dense, c->eval_grid, c->partial, c->stream), "objective kernel");
    CK(launch_objective_finish(c->partial, c->eval_grid, 1.0 / (double)c->n, c->lambda, c->dout, c->stream),
       "objective finish");
    c->launches += 2;
    return ASAGA_OK;
}

// Recomputes abar from alpha in float64; max drift lands in c->dout[1].
asaga_status enqueue_recompute(asaga_ctx *c, std::string *err) {
    const EvalParams e = eval_params(c);
    CK(cudaMemsetAsync(c->acc64, 0, c->d * sizeof(double), c->stream), "memset");
    CK(launch_scatter_rows(e, c->layout, c->dense, 1, c->eval_grid, c->acc64, c->stream), "abar scatter");
    CK(launch_column_finish(e, 1, c->eval_grid, c->acc64, c->partial, c->stream), "abar finish");
    CK(launch_reduce_partials(c->partial, c->eval_grid, 1, c->dout + 1, c->stream), "abar reduce");
    c->launches += 3;
    return ASAGA_OK;
}

asaga_status stream_sync(asaga_ctx *c, std::string *err) {
    CK(cudaStreamSynchronize(c->stream), "stream synchronize");
    return ASAGA_OK;
}

// The most frequent columns (at most kMaxHot, each in at least
// max(64, n/4096) rows) get a per-block shared-memory accumulator in the
// float64 A^T w scatters, where their atomics would otherwise serialise at
// one L2 line.
asaga_status select_hot_columns(asaga_ctx *c, const std::vector<int> &count, std::string *err) {
    const int64_t floor_count = std::max<int64_t>(64, c->n / 4096);
    std::vector<int> cand;
    for (int64_t v = 0; v < c->d; ++v)
        if (count[v] >= floor_count) cand.push_back((int)v);
    std::sort(cand.begin(), cand.end(), [&](int a, int b) { return count[a] != count[b] ? count[a] > count[b] : a < b; });
    if ((int)cand.size() > kMaxHot) cand.resize(kMaxHot);
    c->n_hot = (int)cand.size();
    if (c->n_hot == 0) return ASAGA_OK;
    std::vector<int> slot(c->d, -1);
    for (int s = 0; s < c->n_hot; ++s) slot[cand[s]] = s;
    TRY(dev_alloc(&c->hot_slot, c->d, c, err, "alloc hot slots"));
    TRY(dev_alloc(&c->hot_col, c->n_hot, c, err, "alloc hot columns"));
    CK(cudaMemcpyAsync(c->hot_slot, slot.data(), c->d * sizeof(int), cudaMemcpyHostToDevice, c->stream), "copy slots");
    // copies from pageable memory: the host vectors may go once the calls return
    CK(cudaMemcpyAsync(c->hot_col, cand.data(), c->n_hot * sizeof(int), cudaMemcpyHostToDevice, c->stream),
       "copy hot columns");
    return ASAGA_OK;
}

// Compact layouts of A, applied after the set-up (D, L and the frequent
// columns are computed on the int32, one-value-per-entry layout).
// rows_constant: whether every row's stored values are equal (binary rows
// scaled to unit norm, for instance).
asaga_status rows_constant(asaga_ctx *c, bool *out, std::string *err) {
    *out = false;
    if (c->dense || c->nnz == 0) return ASAGA_OK;
    int *flag = nullptr;
    CK(cudaMallocAsync((void **)&flag, sizeof(int), c->stream), "alloc flag");
    CK(cudaMemsetAsync(flag, 0, sizeof(int), c->stream), "memset flag");
    CK(launch_row_constant_check(c->row_ptr, c->values, c->vtype, c->n, flag, c->stream), "row check");
    ++c->launches;
    CK(cudaMemcpyAsync(c->hstatus, flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "copy flag");
    CK(cudaFreeAsync(flag, c->stream), "free flag");
    TRY(stream_sync(c, err));
    *out = c->hstatus[0] == 0;
    c->hstatus[0] = 0;
    return ASAGA_OK;
}

// rows_equal: keep one float32 value per row (the stored value, exactly)
// instead of one per entry; idx16: uint16 column indices (d <= 65536).  The
// arithmetic is unchanged: the kernels see the same numbers.
asaga_status apply_compact(asaga_ctx *c, bool rows_equal, bool idx16, std::string *err) {
    if (c->dense || c->nnz == 0) return ASAGA_OK;
    const size_t vsz = c->vtype == kF32 ? 4 : 2;
    if (rows_equal) {
        TRY(dev_alloc(&c->row_scale, c->n, c, err, "alloc row values"));
        CK(launch_row_scale(c->row_ptr, c->values, c->vtype, c->n, c->row_scale, c->stream), "row values");
        ++c->launches;
        TRY(stream_sync(c, err));
        cudaFree(c->values);
        c->values = nullptr;
        c->device_bytes -= (int64_t)(c->nnz * vsz + 64);
        c->layout = kRowScale;
    }
    if (idx16 && c->d <= 65536) {
        // 64 bytes of slack: the update kernel copies row slices rounded out to 16-byte boundaries
        TRY(dev_alloc(&c->col16, (size_t)c->nnz + 32, c, err, "alloc 16-bit columns"));
        CK(launch_cols_to_u16(c->col_idx, c->col16, c->nnz, c->stream), "16-bit columns");
        ++c->launches;
        TRY(stream_sync(c, err));
        cudaFree(c->col_idx);
        c->col_idx = nullptr;
        c->device_bytes -= (int64_t)((c->nnz + 4) * sizeof(int32_t));
        c->layout |= kIdx16;
    }
    return ASAGA_OK;
}

// Device set-up, allocations and the copies of the problem: nothing here
// reads the data by its content (no kernel indexes by a column), so it may
// run while the content check is still going on.
asaga_status create_buffers(asaga_ctx *c, const asaga_problem *p, const asaga_options *o, std::string *err) {
    CK(cudaGetDevice(&c->device), "cudaGetDevice");
    cudaDeviceProp prop;
    CK(cudaGetDeviceProperties(&prop, c->device), "cudaGetDeviceProperties");
    c->sms = prop.multiProcessorCount;
    if (o->cuda_stream) {
        c->stream = (cudaStream_t)o->cuda_stream;
    } else {
        CK(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking), "cudaStreamCreate");
        c->own_stream = true;
    }
    for (auto &ev : c->ev) CK(cudaEventCreate(&ev), "cudaEventCreate");

    c->n = p->n;
    c->d = p->d;
    c->dense = p->dense != 0;
    c->nnz = c->dense ? p->n * p->d : p->nnz;
    c->loss = o->loss;
    c->vtype = o->storage_dtype == ASAGA_F32 ? kF32 : (o->storage_dtype == ASAGA_BF16 ? kBF16 : kF16);
    c->lambda = o->lambda;
    c->deterministic = o->deterministic != 0;
    c->plain_writes = o->plain_writes != 0;
    c->sampling = o->sampling;
    c->seed = o->seed;
    c->epochs_per_segment = o->epochs_per_segment > 0 ? o->epochs_per_segment : 1;
    c->abar_every = o->abar_recompute_every;
    c->timeout_s = o->timeout_s;
    c->stride = o->column_stride > 0 ? o->column_stride : (c->d <= 1024 ? 16 : 1);  // 16 float2s = 128 bytes

    const size_t vsz_in = dtype_size(p->values_dtype);
    const size_t vsz = c->vtype == kF32 ? 4 : 2;
    const cudaMemcpyKind kind = p->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;

    // problem
    if (!c->dense) {
        TRY(dev_alloc(&c->row_ptr, c->n + 1, c, err, "alloc row_ptr"));
        // 16 bytes of slack: the update kernel copies row slices rounded out to 16-byte boundaries
        TRY(dev_alloc(&c->col_idx, c->nnz + 4, c, err, "alloc col_idx"));
        CK(cudaMemcpyAsync(c->row_ptr, p->row_ptr, (c->n + 1) * sizeof(int64_t), kind, c->stream), "copy row_ptr");
        if (c->nnz > 0)
            CK(cudaMemcpyAsync(c->col_idx, p->col_idx, c->nnz * sizeof(int32_t), kind, c->stream), "copy col_idx");
    }
    unsigned char *vals = nullptr;
    // 64 bytes of slack: the update kernel copies row slices rounded out to 16-byte boundaries
    TRY(dev_alloc(&vals, (size_t)c->nnz * vsz + 64, c, err, "alloc values"));
    c->values = vals;
    const int in_dt = (int)p->values_dtype;
    const int want_dt = (int)o->storage_dtype;
    if (c->nnz > 0) {
        if (in_dt == want_dt) {
            CK(cudaMemcpyAsync(c->values, p->values, (size_t)c->nnz * vsz, kind, c->stream), "copy values");
        } else {
            const void *src = p->values;
            void *staging = nullptr;
            if (!p->on_device) {
                CK(cudaMallocAsync(&staging, (size_t)c->nnz * vsz_in, c->stream), "alloc staging");
                CK(cudaMemcpyAsync(staging, p->values, (size_t)c->nnz * vsz_in, cudaMemcpyHostToDevice, c->stream),
                   "copy values");
                src = staging;
            }
            cudaError_t e = launch_convert(src, in_dt, c->values, c->vtype, c->nnz, c->stream);
            ++c->launches;
            if (staging) cudaFreeAsync(staging, c->stream);
            if (e != cudaSuccess) return cuda_fail(err, e, "convert values");
        }
    }
    TRY(dev_alloc(&c->lab64, c->n, c, err, "alloc labels"));
    TRY(dev_alloc(&c->lab32, c->n, c, err, "alloc labels"));
    CK(cudaMemcpyAsync(c->lab64, p->labels, c->n * sizeof(double), kind, c->stream), "copy labels");
    CK(launch_labels(c->lab64, c->lab32, c->n, c->stream), "labels kernel");

    // state
    TRY(dev_alloc(&c->alpha, c->n, c, err, "alloc alpha"));
    CK(cudaMemsetAsync(c->alpha, 0, c->n * sizeof(float), c->stream), "memset alpha");
    TRY(dev_alloc(&c->state, (size_t)c->d * c->stride, c, err, "alloc state"));
    CK(cudaMemsetAsync(c->state, 0, (size_t)c->d * c->stride * sizeof(float2), c->stream), "memset state");
    TRY(dev_alloc(&c->dcol, (size_t)c->d, c, err, "alloc D"));
    CK(cudaMemsetAsync(c->dcol, 0, (size_t)c->d * sizeof(float), c->stream), "memset D");
    TRY(dev_alloc(&c->acc64, c->d, c, err, "alloc scratch"));
    c->eval_grid = c->sms * 4;
    if (c->eval_grid > kMaxPartials) c->eval_grid = kMaxPartials;
    TRY(dev_alloc(&c->partial, 2 * (size_t)kMaxPartials, c, err, "alloc partials"));
    TRY(dev_alloc(&c->dout, 8, c, err, "alloc out"));
    TRY(dev_alloc(&c->status, 4, c, err, "alloc status"));
    CK(cudaMallocHost((void **)&c->hout, 8 * sizeof(double)), "alloc pinned");
    CK(cudaMallocHost((void **)&c->hstatus, 4 * sizeof(int)), "alloc pinned");
    CK(cudaHostAlloc((void **)&c->h_cancel, sizeof(int), cudaHostAllocMapped), "alloc cancel flag");
    *c->h_cancel = 0;
    CK(cudaHostGetDevicePointer((void **)&c->d_cancel, c->h_cancel, 0), "cancel flag address");

    return ASAGA_OK;
}

// D from the column counts, L, gamma and the frequent columns of the
// evaluation kernels.  Safe on a problem not yet checked: the kernels skip
// out-of-range columns and row ranges.
asaga_status create_setup(asaga_ctx *c, const asaga_options *o, std::string *err) {
    // D from the column counts (Sec. 2); dense rows give D = 1
    int *count = nullptr;
    std::vector<int> count_h;
    if (!c->dense) {
        CK(cudaMallocAsync((void **)&count, c->d * sizeof(int), c->stream), "alloc counts");
        CK(cudaMemsetAsync(count, 0, c->d * sizeof(int), c->stream), "memset counts");
        CK(launch_count_columns(c->col_idx, c->nnz, c->d, count, c->stream), "count kernel");
        ++c->launches;
    }
    CK(launch_init_state(c->state, c->dcol, c->stride, c->d, count, c->n, c->stream), "init state");
    ++c->launches;
    if (count) {
        count_h.resize(c->d);
        CK(cudaMemcpyAsync(count_h.data(), count, c->d * sizeof(int), cudaMemcpyDeviceToHost, c->stream),
           "copy counts");
        CK(cudaFreeAsync(count, c->stream), "free counts");
    }
    // L = max_i (c |a_i|^2 + lambda max_{v in S_i} D_v) on the stored values
    const double cl = c->loss == ASAGA_LOSS_LOGISTIC ? 0.25 : 1.0;
    const EvalParams e = eval_params(c);
    CK(launch_max_row_smoothness(e, c->nnz, c->vtype, c->dense, cl, c->eval_grid, c->partial, c->dout, c->stream),
       "smoothness kernel");
    c->launches += 2;
    CK(cudaMemcpyAsync(c->hout, c->dout, sizeof(double), cudaMemcpyDeviceToHost, c->stream), "copy L");
    TRY(stream_sync(c, err));
    c->L = c->hout[0] > 0 ? c->hout[0] : (c->lambda > 0 ? c->lambda : 1.0);
    c->gamma = o->gamma > 0 ? o->gamma : (c->L > 0 ? 1.0 / (3.0 * c->L) : 1.0);
    if (c->dense) {
        c->delta = 1.0;
    } else {
        int mx = 0;
        for (int v : count_h) mx = v > mx ? v : mx;
        c->delta = (double)mx / (double)c->n;
    }
    if (!c->dense) TRY(select_hot_columns(c, count_h, err));
    return ASAGA_OK;
}

// The content check of a problem in host memory, on its own thread while
// create_buffers allocates and copies; joined (also on every early return)
// before anything reads the data by content.
struct ContentCheck {
    std::thread th;
    asaga_status status = ASAGA_OK;
    std::string msg;
    int64_t max_row_len = 0;
    void start(const asaga_problem *p, const asaga_options *o) {
        try {
            th = std::thread([this, p, o] { status = validate_content(p, o, &max_row_len, &msg); });
        } catch (const std::system_error &) {  // no thread to be had: check on this one
            status = validate_content(p, o, &max_row_len, &msg);
        }
    }
    void join() {
        if (th.joinable()) th.join();
    }
    ~ContentCheck() { join(); }
};

asaga_status create_impl(asaga_ctx *c, const asaga_problem *p, const asaga_options *o, std::string *err) {
    NvtxRange range("asaga_create");
    TRY(validate_args(p, o, err));
    int64_t mrl = 0;
    ContentCheck check;
    if (p->on_device) {
        TRY(validate_content(p, o, &mrl, err));  // reads device memory: before the set-up
    } else {
        check.start(p, o);
    }
    // The set-up kernels bound every index they read, so they run on the
    // copied problem while the content check is still looking at it; a
    // problem that the check rejects only leaves results that are dropped.
    asaga_status made = create_buffers(c, p, o, err);
    if (made == ASAGA_OK) made = create_setup(c, o, err);
    if (!p->on_device) {
        check.join();
        // a bad problem is reported as such, even when the device set-up failed too
        if (check.status != ASAGA_OK) return fail(err, check.status, check.msg);
        mrl = check.max_row_len;
    }
    if (made != ASAGA_OK) return made;
    c->max_row_len = mrl;
    c->layout = c->vtype;
    if (o->compact && !c->dense) {
        bool rows_equal = false;
        TRY(rows_constant(c, &rows_equal, err));
        TRY(apply_compact(c, rows_equal, c->d <= 65536, err));
    }

    // concurrency: resident warps of the update kernel, bounded by n so that
    // the overlap stays far below n/10 (Theorem 2's condition)
    const int bps = update_max_blocks_per_sm(c->layout, c->dense);
    const int64_t resident = (int64_t)c->sms * bps * (kUpdateBlock / 32);
    int64_t w = o->max_warps > 0 ? o->max_warps : std::max<int64_t>(1, c->n / 64);
    if (w > resident) w = resident;
    if (c->deterministic) w = 1;
    c->warps = (int)w;
    c->resident_warps = (int)resident;
    c->gamma_base = c->gamma;
    return ASAGA_OK;
}

void release(asaga_ctx *c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    cudaFree(c->row_ptr);
    cudaFree(c->col_idx);
    cudaFree(c->col16);
    cudaFree(c->values);
    cudaFree(c->row_scale);
    cudaFree(c->lab32);
    cudaFree(c->lab64);
    cudaFree(c->alpha);
    cudaFree(c->state);
    cudaFree(c->dcol);
    cudaFree(c->acc64);
    cudaFree(c->partial);
    cudaFree(c->dout);
    cudaFree(c->status);
    cudaFree(c->idx_buf);
    cudaFree(c->hot_slot);
    cudaFree(c->hot_col);
    cudaFree(c->long_bits);
    cudaFree(c->d_sums);
    cudaFree(c->tail_c);
    if (c->hout) cudaFreeHost(c->hout);
    if (c->hstatus) cudaFreeHost(c->hstatus);
    if (c->h_cancel) cudaFreeHost(c->h_cancel);
    for (auto &ev : c->ev)
        if (ev) cudaEventDestroy(ev);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    cudaGetLastError();
    delete c;
}

UpdateParams update_params(const asaga_ctx *c) {
    UpdateParams u;
    std::memset(&u, 0, sizeof(u));
    u.n = c->n;
    u.d = c->d;
    u.nnz = c->nnz;
    u.row_ptr = c->row_ptr;
    u.col_idx = layout_cols(c);
    u.values = layout_values(c);
    u.labels = c->lab32;
    u.alpha = c->alpha;
    u.state = c->state;
    u.dcol = c->dcol;
    u.stride = c->stride;
    u.loss = c->loss;
    u.gamma = (float)c->gamma;
    u.lambda = (float)c->lambda;
    u.inv_n = (float)(1.0 / (double)c->n);
    u.seed = c->seed;
    u.t_begin = 0;
    u.count = 0;
    u.short_cores = c->warps;  // concurrent updates; split between the row paths at launch
    u.long_cores = 0;
    u.group = 1;
    u.threshold = -1;
    u.wpb = 1;
    u.short_blocks = 0;
    u.long_bits = nullptr;
    u.tail_c = nullptr;
    u.tail_stride = 0;
    u.idx = nullptr;
    u.fence_each = c->warps == 1 ? 1 : 0;
    u.plain_writes = c->plain_writes ? 1 : 0;
    u.draw_ahead = c->draw_ahead;
    u.sampling = c->sampling;
    u.deadline_ns = 0;
    u.status = c->status;
    u.trace = nullptr;
    u.cancel = nullptr;  // only asaga_run honours asaga_cancel
    return u;
}

// Bits of the rows longer than `threshold` entries and the share of the
// nonzeros they hold (built once per threshold).
asaga_status ensure_row_classes(asaga_ctx *c, int64_t threshold, std::string *err) {
    if (c->bits_threshold == threshold && c->long_bits) return ASAGA_OK;
    if (c->dense) {  // every row has d entries
        c->long_share = c->d > threshold ? 1.0 : 0.0;
        c->bits_threshold = threshold;
        return ASAGA_OK;
    }
    if (!c->long_bits) TRY(dev_alloc(&c->long_bits, (size_t)((c->n + 31) / 32), c, err, "alloc row classes"));
    if (!c->d_sums) TRY(dev_alloc(&c->d_sums, 2, c, err, "alloc row class sums"));
    CK(cudaMemsetAsync(c->d_sums, 0, 2 * sizeof(unsigned long long), c->stream), "memset");
    CK(launch_row_classes(c->row_ptr, c->n, threshold, c->long_bits, c->d_sums, c->stream), "row classes");
    ++c->launches;
    unsigned long long h[2] = {0, 0};
    CK(cudaMemcpyAsync(h, c->d_sums, sizeof(h), cudaMemcpyDeviceToHost, c->stream), "copy row class sums");
    TRY(stream_sync(c, err));
    c->long_share = c->nnz > 0 ? (double)h[0] / (double)c->nnz : 0.0;
    c->bits_threshold = threshold;
    return ASAGA_OK;
}

// How a launch of W warps is laid out on the device: the split of the
// warps between single-warp and multi-warp cores, the block shape and the
// scratch for entries past the register slots.
struct CoreLayout {
    int short_cores = 0, long_cores = 0, group = 1, wpb = 8, short_blocks = 0, grid = 0;
    int64_t threshold = -1;
    int64_t tail_stride = 0;
    bool both = false;  // both paths in use (the row classes decide)
};

// Layout of W warps under the row path (threshold, group).  The row path
// regroups the warps into cores and keeps their number: measured on a
// GB300, the stability frontier of the asynchronous iteration lies at a
// product of total warps and step, not of concurrent updates (cores of 4
// warps at the cores x step of a converging single-warp run stalled on a
// plateau; at the same warps x step they converged).  With both paths the
// long rows' cores get the share of the warps that their rows hold of the
// nonzeros (long_share; ensure_row_classes must have run).  serial: one
// core, strictly in order (only one path can then apply).
CoreLayout core_layout(const asaga_ctx *c, int W, int64_t threshold, int group, bool serial) {
    CoreLayout L;
    if (group <= 1 || threshold >= c->max_row_len) threshold = -1;  // no row takes the multi-warp path
    if (serial && threshold > 0) threshold = -1;
    if (threshold > 0 && W < group + 1) threshold = -1;
    L.threshold = threshold;
    L.group = threshold < 0 ? 1 : group;
    const int G = L.group;
    if (threshold < 0) {
        L.short_cores = W;
    } else if (threshold == 0) {
        L.long_cores = serial ? 1 : std::max(1, W / G);
    } else {
        L.both = true;
        int wl = (int)std::llround((double)W * c->long_share);
        wl = std::max(G, std::min(W - 1, wl));
        L.long_cores = std::max(1, wl / G);
        L.short_cores = std::max(1, W - L.long_cores * G);
    }
    const int warps = L.short_cores + L.long_cores * G;
    const int per_sm = (warps + c->sms - 1) / std::max(1, c->sms);
    int wpb = warps <= 1 ? 1 : (c->spread ? std::min(kUpdateBlock / 32, std::max(1, per_sm)) : kUpdateBlock / 32);
    wpb = std::max(wpb, G);
    wpb = (wpb + G - 1) / G * G;
    if (L.short_cores + L.long_cores <= 1) wpb = G;  // one core
    L.wpb = wpb;
    L.short_blocks = (L.short_cores + wpb - 1) / wpb;
    const int cpb = wpb / G;
    L.grid = L.short_blocks + (L.long_cores + cpb - 1) / cpb;
    // register capacity of a core: 32 x warps x slots entries
    const int slots = update_register_slots(c->dense, false);
    int64_t need = 0;
    if (L.short_cores > 0) {
        const int64_t longest = L.threshold > 0 ? std::min(L.threshold, c->max_row_len) : c->max_row_len;
        need = std::max<int64_t>(need, longest - 32 * slots);
    }
    if (L.long_cores > 0) need = std::max<int64_t>(need, c->max_row_len - (int64_t)32 * G * slots);
    L.tail_stride = need;
    return L;
}

int update_warps_per_block(const asaga_ctx *c, int nwarps) {
    return core_layout(c, nwarps, c->row_threshold, c->row_group, nwarps <= 1).wpb;
}

// Launches the updates on u.short_cores warps (the callers' "warps"),
// grouped into cores by the context's row path, in its block shape.
asaga_status launch_updates(asaga_ctx *c, UpdateParams u, std::string *err) {
    // eight warps to a block, or (c->spread) the warps spread evenly over
    // the SMs, one block per SM while they allow: then each SM's load/store
    // units and outstanding misses serve fewer warps, which helps a
    // latency-bound state larger than L2 and not a small hot-line-bound one
    // (the autotuner times both)
    const int C = u.short_cores;
    const bool serial = u.fence_each != 0 || u.idx != nullptr;
    const CoreLayout L = core_layout(c, C, c->row_threshold, c->row_group, serial);
    if (L.both) TRY(ensure_row_classes(c, L.threshold, err));
    const CoreLayout M = L.both ? core_layout(c, C, c->row_threshold, c->row_group, serial) : L;  // with the share
    u.short_cores = M.short_cores;
    u.long_cores = M.long_cores;
    u.group = M.group;
    u.threshold = M.threshold;
    u.wpb = M.wpb;
    u.short_blocks = M.short_blocks;
    u.long_bits = M.both ? c->long_bits : nullptr;
    if (M.tail_stride > 0) {
        const int64_t need = (int64_t)(M.short_cores + M.long_cores) * M.tail_stride;
        if (need > c->tail_floats) {
            CK(cudaStreamSynchronize(c->stream), "sync");
            if (c->tail_c) {
                cudaFree(c->tail_c);
                c->device_bytes -= c->tail_floats * (int64_t)sizeof(float);
                c->tail_c = nullptr;
                c->tail_floats = 0;
            }
            TRY(dev_alloc(&c->tail_c, (size_t)need, c, err, "alloc row tail scratch"));
            c->tail_floats = need;
        }
        u.tail_c = c->tail_c;
        u.tail_stride = M.tail_stride;
    }
    CK(launch_update(u, c->layout, c->dense, M.grid, c->stream), "update kernel");
    ++c->launches;
    return ASAGA_OK;
}

asaga_status run_impl(asaga_ctx *c, double max_epochs, double target, double f_star, asaga_result *res,
                      std::string *err) {
    if (!(max_epochs >= 0) || !std::isfinite(max_epochs)) return fail(err, ASAGA_EINVAL, "max_epochs must be >= 0");
    if (!std::isfinite(target)) return fail(err, ASAGA_EINVAL, "target must be finite");
    if (target > 0 && (!std::isfinite(f_star) || f_star == 0.0))
        return fail(err, ASAGA_EINVAL, "f_star must be finite and nonzero when a target is set");
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    const auto t0 = std::chrono::steady_clock::now();
    asaga_result r;
    std::memset(&r, 0, sizeof(r));
    r.f_last = NAN;
    r.rel_subopt = NAN;
    const int64_t launches0 = c->launches;
    CK(cudaMemsetAsync(c->status, 0, sizeof(int), c->stream), "memset status");
    __atomic_store_n(c->h_cancel, 0, __ATOMIC_SEQ_CST);
    double epochs_done = 0;
    asaga_status st = target > 0 ? ASAGA_ENOTCONVERGED : ASAGA_OK;
    int64_t seg = 0;
    while (epochs_done < max_epochs) {
        NvtxRange range("asaga_run segment");
        if (__atomic_load_n(c->h_cancel, __ATOMIC_SEQ_CST)) {  // requested between segments
            st = ASAGA_ECANCELLED;
            fail(err, st, "cancelled");
            break;
        }
        const double ep = std::min((double)c->epochs_per_segment, max_epochs - epochs_done);
        const int64_t count = (int64_t)std::llround(ep * (double)c->n);
        UpdateParams u = update_params(c);
        u.t_begin = (uint64_t)c->updates_done;
        u.count = count;
        u.cancel = c->d_cancel;
        if (c->timeout_s > 0) {
            const double left = c->timeout_s -
                                std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            u.deadline_ns = left > 0 ? (uint64_t)(left * 1e9) : 1;
        }
        CK(cudaEventRecord(c->ev[0], c->stream), "event");
        if (count > 0) TRY(launch_updates(c, u, err));
        CK(cudaEventRecord(c->ev[1], c->stream), "event");
        ++seg;
        // every abar_every-th segment of the context, counted across calls
        const bool recompute = c->abar_every > 0 && ++c->segments_done % c->abar_every == 0;
        if (recompute) TRY(enqueue_recompute(c, err));
        TRY(enqueue_objective(c, err));
        CK(cudaEventRecord(c->ev[2], c->stream), "event");
        CK(cudaMemcpyAsync(c->hout, c->dout, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream), "copy f");
        CK(cudaMemcpyAsync(c->hstatus, c->status, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "copy status");
        TRY(stream_sync(c, err));
        float ms_solve = 0, ms_eval = 0;
        cudaEventElapsedTime(&ms_solve, c->ev[0], c->ev[1]);
        cudaEventElapsedTime(&ms_eval, c->ev[1], c->ev[2]);
        r.solver_seconds += ms_solve * 1e-3;
        r.eval_seconds += ms_eval * 1e-3;
        c->updates_done += count;
        r.updates += count;
        epochs_done += ep;
        r.segments = seg;
        r.f_last = c->hout[0];
        if (recompute) r.abar_drift = c->hout[1];
        if (target > 0 || std::isfinite(f_star)) r.rel_subopt = (r.f_last - f_star) / std::fabs(f_star);
        if (*c->hstatus & 4) {
            st = ASAGA_ECUDA;
            fail(err, st, "update kernel found a malformed row range");
            break;
        }
        if (*c->hstatus & 48) {
            st = ASAGA_ECUDA;
            fail(err, st, (*c->hstatus & 16) ? "update kernel: a row's staging copy did not complete in time"
                                             : "update kernel: row scratch smaller than a row");
            break;
        }
        if (*c->hstatus & 1) {
            st = ASAGA_ETIMEOUT;
            fail(err, st, "timeout");
            break;
        }
        if (*c->hstatus & 8) {
            st = ASAGA_ECANCELLED;
            fail(err, st, "cancelled");
            break;
        }
        if (!std::isfinite(r.f_last)) {
            st = ASAGA_EDIVERGED;
            fail(err, st, "objective is not finite");
            break;
        }
        if (target > 0 && r.rel_subopt <= target) {
            st = ASAGA_OK;
            break;
        }
    }
    if (seg == 0) {  // max_epochs == 0: report f at the current iterate
        TRY(enqueue_objective(c, err));
        CK(cudaMemcpyAsync(c->hout, c->dout, sizeof(double), cudaMemcpyDeviceToHost, c->stream), "copy f");
        TRY(stream_sync(c, err));
        r.f_last = c->hout[0];
        if (std::isfinite(f_star) && f_star != 0) r.rel_subopt = (r.f_last - f_star) / std::fabs(f_star);
        if (target > 0 && r.rel_subopt <= target) st = ASAGA_OK;
    }
    r.epochs = epochs_done;
    r.kernel_launches = c->launches - launches0;
    r.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (res) *res = r;
    if (st == ASAGA_ENOTCONVERGED) fail(err, st, "max_epochs reached before the target");
    return st;
}

asaga_status reset_state(asaga_ctx *c, std::string *err) {
    CK(cudaMemsetAsync(c->alpha, 0, c->n * sizeof(float), c->stream), "memset alpha");
    CK(cudaMemset2DAsync(c->state, (size_t)c->stride * sizeof(float2), 0, sizeof(float2), c->d, c->stream),
       "memset state");
    c->updates_done = 0;
    c->segments_done = 0;
    return ASAGA_OK;
}

asaga_status enqueue_grad(asaga_ctx *c, std::string *err) {
    const EvalParams e = eval_params(c);
    CK(cudaMemsetAsync(c->acc64, 0, c->d * sizeof(double), c->stream), "memset");
    CK(launch_scatter_rows(e, c->layout, c->dense, 0, c->eval_grid, c->acc64, c->stream), "gradient scatter");
    CK(launch_column_finish(e, 0, c->eval_grid, c->acc64, c->partial, c->stream), "gradient finish");
    CK(launch_reduce_partials(c->partial, c->eval_grid, 0, c->dout + 2, c->stream), "gradient reduce");
    c->launches += 3;
    return ASAGA_OK;
}

// One epoch of updates with the given warps and step; returns the update
// kernel's device time and |grad f|^2 after it.
asaga_status trial_epoch(asaga_ctx *c, int warps, double gamma, double *ms, double *g2, std::string *err) {
    UpdateParams u = update_params(c);
    u.short_cores = warps;
    u.fence_each = warps == 1;
    u.gamma = (float)gamma;
    u.t_begin = (uint64_t)c->updates_done;
    u.count = c->n;
    CK(cudaMemsetAsync(c->status, 0, sizeof(int), c->stream), "memset status");
    CK(cudaEventRecord(c->ev[0], c->stream), "event");
    TRY(launch_updates(c, u, err));
    CK(cudaEventRecord(c->ev[1], c->stream), "event");
    c->updates_done += c->n;
    if (g2) {
        TRY(enqueue_grad(c, err));
        CK(cudaMemcpyAsync(c->hout + 2, c->dout + 2, sizeof(double), cudaMemcpyDeviceToHost, c->stream), "copy");
    }
    CK(cudaMemcpyAsync(c->hstatus, c->status, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "copy status");
    TRY(stream_sync(c, err));
    if (*c->hstatus & 52) return fail(err, ASAGA_ECUDA, "update kernel status " + std::to_string(*c->hstatus));
    float f = 0;
    cudaEventElapsedTime(&f, c->ev[0], c->ev[1]);
    *ms = f;
    if (g2) *g2 = c->hout[2];
    return ASAGA_OK;
}

// ---------------------------------------------------------------------------
// Autotuner.  Measured behaviour of asynchronous Sparse SAGA on a GB300 that
// it relies on:
//  * warps x step has a stability frontier: above it the iterate does not
//    converge (logistic: |grad f|^2 bounces on a plateau; squared loss:
//    divergence), below it the run converges, and near it the outcome
//    varies from run to run;
//  * below the frontier the epochs needed depend on the step, not on the
//    number of warps;
//  * the epoch time falls with the number of warps until the kernel saturates.
// So the frontier is located at one warp count, and warp counts are then
// raced along warps x step = constant, one notch inside the frontier.

// The trial records and the decision rules on them (trend, convergence,
// predicted epochs) are host-only and tested on the CPU.
using namespace asaga::tune;

// update time a race trial may spend beyond its first trial_epochs epochs
constexpr double kTuneExtendMs = 250.0;
// predicted-time tolerance in favour of fewer warps (and larger steps)
constexpr double kTuneFewerWarps = 1.2;

// Trial epochs at (W, gamma), appended to t: |grad f|^2 after each.  Stops
// early on divergence, on reaching stop_level, or once the trial's update
// time exceeds give_up_ms.
asaga_status trial_epochs_run(asaga_ctx *c, int W, double gamma, double g0, int E, double stop_level,
                              double give_up_ms, TuneTrial *t, std::string *err) {
    for (int e = 0; e < E && !t->diverged; ++e) {
        double ms = 0, g = 0;
        TRY(trial_epoch(c, W, gamma, &ms, &g, err));
        t->t_ms += ms;
        t->epochs += 1;
        if (!std::isfinite(g) || g > 1e6 * g0) {
            t->diverged = true;
            break;
        }
        t->y.push_back(std::log10(std::max(g / g0, 1e-300)));
        if (t->y.back() <= stop_level || t->t_ms > give_up_ms) break;
    }
    return ASAGA_OK;
}

// One trial: from x = 0, up to E epochs (see trial_epochs_run).
asaga_status tune_trial(asaga_ctx *c, int W, double gamma, double g0, int E, double stop_level, double give_up_ms,
                        TuneTrial *out, std::string *err) {
    TRY(reset_state(c, err));
    *out = TuneTrial();
    return trial_epochs_run(c, W, gamma, g0, E, stop_level, give_up_ms, out, err);
}

// Row paths worth timing for a problem: multi-warp cores of G = 2, 4, 8
// warps, for every row (T = 0) when the mean row fills the G warps' lanes,
// or for the rows longer than T = 128, 256, 512 entries when those hold at
// least 2% of the nonzeros.
asaga_status row_path_candidates(asaga_ctx *c, std::vector<std::pair<int64_t, int>> *out, std::string *err) {
    out->clear();
    const double mean_len = c->n > 0 ? (double)c->nnz / (double)c->n : 0.0;
    for (int G : {2, 4, 8}) {
        if ((int64_t)32 * G > c->max_row_len) continue;
        if (mean_len >= 32.0 * G) out->push_back({0, G});
        if (c->dense) continue;
        for (int64_t T : {128, 256, 512}) {
            if (T >= c->max_row_len || T < 32 * G) continue;
            TRY(ensure_row_classes(c, T, err));
            if (c->long_share < 0.02) continue;
            out->push_back({T, G});
        }
    }
    return ASAGA_OK;
}

// Epoch time of the row path (T, G) at (warps, gamma): the faster of two
// epochs after one untimed, from x = 0.
asaga_status time_row_path(asaga_ctx *c, int warps, double gamma, int64_t T, int G, double *ms_out, double *seconds,
                           std::string *err) {
    c->row_threshold = T;
    c->row_group = G;
    TRY(reset_state(c, err));
    double best = INFINITY;
    for (int e = 0; e < 3; ++e) {
        double ms = 0;
        TRY(trial_epoch(c, warps, gamma, &ms, nullptr, err));
        *seconds += ms * 1e-3;
        if (e > 0) best = std::min(best, ms);
    }
    *ms_out = best;
    return ASAGA_OK;
}

asaga_status autotune_impl(asaga_ctx *c, double trial_epochs, asaga_tune_result *res, std::string *err) {
    NvtxRange range("asaga_autotune");
    if (c->deterministic) return fail(err, ASAGA_EINVAL, "autotune needs asynchronous mode");
    if (!std::isfinite(trial_epochs)) return fail(err, ASAGA_EINVAL, "trial_epochs must be finite");
    c->row_threshold = -1;  // the trials run on single-warp cores; the row path comes last
    c->row_group = 1;
    c->draw_ahead = 0;      // and the draw placement after it
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    const int E_race = trial_epochs > 0 ? std::max(4, (int)std::ceil(trial_epochs)) : 24;
    const int E_probe = std::min(16, E_race);
    // steps gamma0 * 2^(-k/2), k in [kTop, kBottom]; the largest, 2^1.5 gamma0 =
    // 0.94/L (gamma0 = 1/(3L)), stays below 1/L, past which a serial run
    // of SAGA is not expected to be stable either
    constexpr int kTop = -3, kBottom = 16;
    auto step = [&](int k) { return c->gamma_base * std::pow(2.0, -0.5 * k); };
    // Theorem 2 wants the overlap tau below n/10; measured, tau is 1.5 to 4
    // times the number of warps: at most n/64 warps keeps tau below n/16
    const int64_t cap = std::max<int64_t>(1, std::min<int64_t>(c->resident_warps, c->n / 64));
    asaga_tune_result r;
    std::memset(&r, 0, sizeof(r));
    r.warps = c->warps;
    r.gamma = c->gamma_base;
    r.score = -1.0;
    TRY(reset_state(c, err));
    TRY(enqueue_grad(c, err));
    CK(cudaMemcpyAsync(c->hout + 2, c->dout + 2, sizeof(double), cudaMemcpyDeviceToHost, c->stream), "copy");
    TRY(stream_sync(c, err));
    const double g0 = c->hout[2];
    if (!(g0 > 0) || !std::isfinite(g0)) {  // x = 0 is already optimal: nothing to tune
        if (res) *res = r;
        return ASAGA_OK;
    }
    auto run = [&](int W, int k, int E, double stop_level, double give_up, TuneTrial *t) -> asaga_status {
        TRY(tune_trial(c, W, step(k), g0, E, stop_level, give_up, t, err));
        ++r.trials;
        r.seconds += t->t_ms * 1e-3;
        return ASAGA_OK;
    };

    // 1. the frontier at a probe warp count: bisection for the largest
    //    converging step (k = kTop - 1 stands for "not converging", kBottom + 1
    //    for "converging"); if no step converges, probe with 8x fewer warps
    int Wp = (int)std::min<int64_t>(cap, 1024);
    int kF = kBottom + 1;
    for (int attempt = 0; attempt < 3; ++attempt) {
        int lo = kTop - 1, hi = kBottom + 1;
        while (hi - lo > 1) {
            const int mid = lo + (hi - lo) / 2;
            TuneTrial t;
            TRY(run(Wp, mid, E_probe, kTuneConverged, INFINITY, &t));
            if (converging(t)) hi = mid;
            else lo = mid;
        }
        kF = hi;
        if (kF <= kBottom || Wp == 1) break;
        Wp = std::max(1, Wp / 8);
    }
    if (kF > kBottom) {  // no step converges visibly within the trials: keep the defaults
        TRY(reset_state(c, err));
        if (res) *res = r;
        return ASAGA_OK;
    }

    // 2. race warp counts Wp * 2^j at k = kF + 2j + 1 (the same warps x step,
    //    one notch inside the frontier; the step never above the ladder's top),
    //    by predicted update time to reach kTuneDeep
    double best_ms = INFINITY;
    double best_pe = INFINITY;  // the winner's predicted epochs
    int best_w = Wp, best_k = std::min(kBottom, kF + 2);  // used if no race trial settles
    auto candidate = [&](int64_t W, int k, bool *improved) -> asaga_status {
        *improved = false;
        if (W < 1 || W > cap || k > kBottom) return ASAGA_OK;
        TuneTrial t;
        const double give_up = std::isfinite(best_ms) ? 1.5 * best_ms : INFINITY;
        TRY(run((int)W, k, E_race, kTuneDeep, give_up, &t));
        // a prediction far beyond the trial extrapolates the early, fast phase
        // of an ill-conditioned problem: run on (up to 8x the epochs, while
        // the trial is cheap) until the prediction is within 2x of its length
        while (!t.diverged && t.epochs < 8 * E_race && t.t_ms < std::min(give_up, kTuneExtendMs)) {
            const double pe = predict_epochs(t);
            if (!std::isfinite(pe) || pe <= 2.0 * t.epochs || t.y.back() <= kTuneDeep) break;
            const double before = t.t_ms;
            TRY(trial_epochs_run(c, (int)W, step(k), g0, std::max(1, t.epochs / 4), kTuneDeep, give_up, &t, err));
            r.seconds += (t.t_ms - before) * 1e-3;
        }
        const double pe = predict_epochs(t);
        const double ms = pe * t.ms_per_epoch();
        // fewer warps and a larger step win within a tolerance: the step
        // carries the slow tail of an ill-conditioned problem beyond the
        // trial, and the overlap tau is smaller
        const bool better = !std::isfinite(best_ms) ? std::isfinite(ms)
                            : W < best_w        ? ms < kTuneFewerWarps * best_ms
                            : W > best_w        ? ms * kTuneFewerWarps < best_ms
                                                : ms < best_ms;
        if (better) {
            best_ms = ms;
            best_pe = pe;
            best_w = (int)W;
            best_k = k;
            *improved = true;
        }
        return ASAGA_OK;
    };
    auto warps_at = [&](int j) -> int64_t { return j >= 0 ? ((int64_t)Wp << j) : ((int64_t)Wp >> -j); };
    auto k_at = [&](int j) { return std::max(kTop, kF + 2 * j + 1); };
    bool improved = false;
    // a frontier read too optimistically leaves every candidate on the
    // plateau: race again one notch further inside (twice at most)
    for (int retry = 0; retry < 3 && !std::isfinite(best_ms); ++retry, ++kF) {
        if (kF + 1 > kBottom) break;
        best_w = Wp;
        best_k = std::min(kBottom, kF + 2);
        TRY(candidate(warps_at(0), k_at(0), &improved));
        for (int j = -1; warps_at(j) >= 1 && k_at(j + 1) > kTop; --j) {  // fewer warps, larger steps
            TRY(candidate(warps_at(j), k_at(j), &improved));
            if (!improved && std::isfinite(best_ms)) break;
        }
        for (int j = 1; warps_at(j) <= cap; ++j) {  // more warps, smaller steps
            TRY(candidate(warps_at(j), k_at(j), &improved));
            if (!improved && std::isfinite(best_ms)) break;
        }
    }
    // 3. at the winning warp count, smaller steps while they are faster (well
    //    conditioned problems need no more than a small step per update)
    const int k_raced = best_k;
    if (std::isfinite(best_ms))
        for (int k = best_k + 1; k <= kBottom; ++k) {
            TRY(candidate(best_w, k, &improved));
            if (!improved) break;
        }
    //    When none was, one notch larger: the race put every warp count one
    //    notch inside the frontier measured at the probe count, and fewer
    //    warps can carry a larger W x gamma than that (measured: URL-shaped
    //    at 256 warps reaches 1e-6 in 14 epochs one notch out, 19 at the raced
    //    step).  Only where the overlap stays far below n (W <= n/256, tau
    //    below n/64): on small problems the larger step was seen to pass the
    //    trials and then stall on a plateau.  The confirmation below still
    //    guards against a late plateau.
    if (std::isfinite(best_ms) && best_k == k_raced && best_k - 1 >= kTop && (int64_t)best_w * 256 <= c->n)
        TRY(candidate(best_w, best_k - 1, &improved));
    // confirmation: the winner over a trial twice as long must still show a
    // downward trend (a plateau can set in after a short trial's early
    // progress); one notch smaller a step while it does not (three times at
    // most).  Where the warps are above n/256 (the overlap a sizeable part of
    // n) a trend is not enough: measured on instances of 55 k and 61 k rows
    // at 431 and 478 warps, tuned schedules passed it and then stalled near
    // 2e-4 for thousands of epochs.  There the trial runs on to 1.5x the
    // winner's predicted epochs and must reach the prediction level, when
    // that prediction is within 8 race lengths (epochs are cheap at such n).
    const bool reach = (int64_t)best_w * 256 > c->n && 1.5 * best_pe <= 8.0 * E_race;
    const int E_confirm = reach ? std::max(2 * E_race, (int)std::ceil(1.5 * best_pe)) : 2 * E_race;
    if (std::isfinite(best_ms))
        for (int attempt = 0; attempt < 3 && best_k <= kBottom; ++attempt) {
            TuneTrial t;
            TRY(run(best_w, best_k, E_confirm, kTuneDeep, std::max(4.0 * kTuneExtendMs, 3.0 * best_ms), &t));
            const bool ok = reach ? !t.diverged && !t.y.empty() && t.y.back() <= kTuneDeep
                                  : !t.diverged && std::isfinite(predict_epochs(t));
            if (ok) break;
            if (best_k == kBottom) break;
            ++best_k;
        }
    // 4. the block shape at the winner: eight warps per block or the warps
    //    spread over the SMs (the faster of two timed epochs each)
    c->spread = false;
    if (std::isfinite(best_ms) && (best_w + c->sms - 1) / std::max(1, c->sms) < kUpdateBlock / 32) {
        double t_shape[2] = {INFINITY, INFINITY};
        for (int shape = 0; shape < 2; ++shape) {
            c->spread = shape == 1;
            TRY(reset_state(c, err));
            for (int e = 0; e < 3; ++e) {
                double ms = 0;
                TRY(trial_epoch(c, best_w, step(best_k), &ms, nullptr, err));
                r.seconds += ms * 1e-3;
                if (e > 0) t_shape[shape] = std::min(t_shape[shape], ms);
            }
        }
        c->spread = t_shape[1] < 0.98 * t_shape[0];
    }
    // 5. the row path at the winner (the same warps and step, regrouped into
    //    cores): rows longer than T entries on cores of G warps, for the
    //    (T, G) of row_path_candidates, timed; the two fastest that beat
    //    single warps by 3% then run a race trial, and the first whose
    //    predicted time beats the winner's by 3% is kept (a plateau has no
    //    prediction)
    c->row_threshold = -1;
    c->row_group = 1;
    if (std::isfinite(best_ms)) {
        std::vector<std::pair<int64_t, int>> cand;
        TRY(row_path_candidates(c, &cand, err));
        if (!cand.empty()) {
            double t_single = INFINITY;
            TRY(time_row_path(c, best_w, step(best_k), -1, 1, &t_single, &r.seconds, err));
            std::vector<std::pair<double, size_t>> order;
            for (size_t j = 0; j < cand.size(); ++j) {
                double t = INFINITY;
                TRY(time_row_path(c, best_w, step(best_k), cand[j].first, cand[j].second, &t, &r.seconds, err));
                if (t < 0.97 * t_single) order.push_back({t, j});
            }
            std::sort(order.begin(), order.end());
            int64_t keep_T = -1;
            int keep_G = 1;
            for (size_t o = 0; o < order.size() && o < 2; ++o) {
                c->row_threshold = cand[order[o].second].first;
                c->row_group = cand[order[o].second].second;
                TuneTrial t;
                TRY(run(best_w, best_k, E_race, kTuneDeep, 1.5 * best_ms, &t));
                const double ms = predict_epochs(t) * t.ms_per_epoch();
                if (!t.diverged && std::isfinite(ms) && ms < 0.97 * best_ms) {
                    keep_T = c->row_threshold;
                    keep_G = c->row_group;
                    best_ms = ms;
                    break;
                }
            }
            c->row_threshold = keep_T;
            c->row_group = keep_G;
        }
    }
    // 6. the draw placement at the winner: the next row drawn inside the
    //    updates' windows hides the sampler's latency but lengthens the
    //    windows (more overlap at the same warps).  Near the frontier that
    //    can turn a converging schedule into one that stalls after a long
    //    downward trend (measured: RCV1-shaped rows at the tuned 512 warps),
    //    so a trend is not enough: each of two trials of twice the race
    //    length must reach the prediction level itself, and the slower must
    //    beat the winner by 3%.  Only where the overlap stays far below n
    //    (W <= n/256), as for the larger step of step 3: on an instance of
    //    55 k rows at 431 warps the trials passed and the run then stalled
    //    at 2e-4 for 3000 epochs.
    if (std::isfinite(best_ms) && (int64_t)best_w * 256 <= c->n) {
        c->draw_ahead = 1;
        double worst = 0;
        for (int trial = 0; trial < 2 && std::isfinite(worst); ++trial) {
            TuneTrial t;
            TRY(run(best_w, best_k, 2 * E_race, kTuneDeep, best_ms, &t));
            const bool deep = !t.diverged && !t.y.empty() && t.y.back() <= kTuneDeep;
            worst = deep ? std::max(worst, t.t_ms) : INFINITY;  // the update time to the level
        }
        if (std::isfinite(worst) && worst < 0.97 * best_ms)
            best_ms = worst;
        else
            c->draw_ahead = 0;
    }
    if (std::isfinite(best_ms)) r.score = 1e3 / best_ms;
    r.warps = best_w;
    r.gamma = step(best_k);
    r.row_threshold = c->row_threshold;
    r.row_group = c->row_group;
    r.draw_ahead = c->draw_ahead;
    TRY(reset_state(c, err));
    c->warps = r.warps;
    c->gamma = r.gamma;
    if (res) *res = r;
    return ASAGA_OK;
}

// Overlap of asynchronous updates (the tau of Assumption 1), measured as in
// App. E.2: for each update, the number of other updates whose processing
// interval (reads issued .. writes issued) intersects its own; tau_paper =
// max over consecutive windows of 100 updates (in start order) of the
// window's average overlap.
asaga_status overlap_impl(asaga_ctx *c, double epochs, asaga_overlap *out, uint64_t *times, int64_t capacity,
                          std::string *err) {
    if (!out) return fail(err, ASAGA_EINVAL, "out is NULL");
    if (!(epochs > 0) || !std::isfinite(epochs)) return fail(err, ASAGA_EINVAL, "epochs must be > 0");
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    const int64_t count = (int64_t)std::llround(epochs * (double)c->n);
    if (count < 2) return fail(err, ASAGA_EINVAL, "need at least 2 updates");
    if (times && capacity < 2 * count)
        return fail(err, ASAGA_EINVAL, "times holds " + std::to_string(capacity) + " values, the trace " +
                                           std::to_string(2 * count));
    uint64_t *trace = nullptr;
    CK(cudaMallocAsync((void **)&trace, 2 * count * sizeof(uint64_t), c->stream), "alloc trace");
    UpdateParams u = update_params(c);
    u.t_begin = (uint64_t)c->updates_done;
    u.count = count;
    u.trace = trace;
    CK(cudaEventRecord(c->ev[0], c->stream), "event");
    asaga_status st = launch_updates(c, u, err);
    CK(cudaEventRecord(c->ev[1], c->stream), "event");
    std::vector<uint64_t> h(2 * count);
    if (st == ASAGA_OK) {
        cudaError_t e = cudaMemcpyAsync(h.data(), trace, 2 * count * sizeof(uint64_t), cudaMemcpyDeviceToHost,
                                        c->stream);
        if (e != cudaSuccess) st = cuda_fail(err, e, "copy trace");
    }
    cudaFreeAsync(trace, c->stream);
    if (st != ASAGA_OK) return st;
    TRY(stream_sync(c, err));
    c->updates_done += count;
    float ms = 0;
    cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]);
    std::vector<uint64_t> starts(count), ends(count);
    std::vector<int64_t> order(count);
    double window_sum = 0;
    for (int64_t t = 0; t < count; ++t) {
        starts[t] = h[2 * t];
        ends[t] = h[2 * t + 1];
        order[t] = t;
        window_sum += (double)(ends[t] - starts[t]);
    }
    if (times) std::copy(h.begin(), h.end(), times);
    // start order; updates that start at the same time stay in update order
    std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return starts[a] < starts[b]; });
    std::vector<uint64_t> s_sorted(starts), e_sorted(ends);
    std::sort(s_sorted.begin(), s_sorted.end());
    std::sort(e_sorted.begin(), e_sorted.end());
    // overlap(t) = #{r != t : start_r <= end_t and end_r >= start_t}
    std::vector<double> ov(count);
    double sum = 0, mx = 0;
    for (int64_t k = 0; k < count; ++k) {
        const int64_t t = order[k];
        const int64_t started = std::upper_bound(s_sorted.begin(), s_sorted.end(), ends[t]) - s_sorted.begin();
        const int64_t finished_before = std::lower_bound(e_sorted.begin(), e_sorted.end(), starts[t]) - e_sorted.begin();
        ov[k] = (double)(started - finished_before - 1);
        sum += ov[k];
        mx = std::max(mx, ov[k]);
    }
    double paper = 0;
    for (int64_t k = 0; k + 100 <= count; k += 100) {
        double w = 0;
        for (int64_t j = k; j < k + 100; ++j) w += ov[j];
        paper = std::max(paper, w / 100.0);
    }
    out->updates = count;
    out->warps = c->warps;
    out->tau_mean = sum / (double)count;
    out->tau_max = mx;
    out->tau_paper = paper;
    out->window_ns_mean = window_sum / (double)count;
    out->seconds = ms * 1e-3;
    return ASAGA_OK;
}

asaga_status run_indices_impl(asaga_ctx *c, const int64_t *idx, int64_t count, int on_device, std::string *err) {
    if (count < 0) return fail(err, ASAGA_EINVAL, "count < 0");
    if (count == 0) return ASAGA_OK;
    if (!idx) return fail(err, ASAGA_EINVAL, "idx is NULL");
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    const int64_t *didx = idx;
    if (!on_device) {
        for (int64_t t = 0; t < count; ++t)
            if (idx[t] < 0 || idx[t] >= c->n) return fail(err, ASAGA_EINVAL, "index out of range at " + std::to_string(t));
        if (count > c->idx_cap) {
            CK(cudaStreamSynchronize(c->stream), "sync");
            if (c->idx_buf) {
                cudaFree(c->idx_buf);
                c->device_bytes -= c->idx_cap * (int64_t)sizeof(int64_t);
                c->idx_buf = nullptr;
                c->idx_cap = 0;
            }
            TRY(dev_alloc(&c->idx_buf, count, c, err, "alloc index buffer"));
            c->idx_cap = count;
        }
        CK(cudaMemcpyAsync(c->idx_buf, idx, count * sizeof(int64_t), cudaMemcpyHostToDevice, c->stream), "copy idx");
        didx = c->idx_buf;
    }
    UpdateParams u = update_params(c);
    u.short_cores = 1;
    u.fence_each = 1;
    u.idx = didx;
    u.count = count;
    CK(cudaMemsetAsync(c->status, 0, sizeof(int), c->stream), "memset status");
    TRY(launch_updates(c, u, err));
    CK(cudaMemcpyAsync(c->hstatus, c->status, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "copy status");
    TRY(stream_sync(c, err));
    if (*c->hstatus & 2) return fail(err, ASAGA_EINVAL, "index out of range in device index array");
    if (*c->hstatus & 52) return fail(err, ASAGA_ECUDA, "update kernel status " + std::to_string(*c->hstatus));
    return ASAGA_OK;
}

// ---------------------------------------------------------------- batches

void batch_release(asaga_batch *b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->graph_rc) cudaGraphExecDestroy(b->graph_rc);
    for (auto *c : b->ctx) release(c);
    cudaFree(b->d_rpartial);
    cudaFree(b->d_drift);
    cudaFree(b->d_status);
    if (b->h_drift) cudaFreeHost(b->h_drift);
    if (b->h_status) cudaFreeHost(b->h_status);
    cudaFree(b->d_up);
    cudaFree(b->d_ev);
    cudaFree(b->d_block_begin);
    cudaFree(b->d_partial);
    cudaFree(b->d_f);
    if (b->h_up) cudaFreeHost(b->h_up);
    if (b->h_f) cudaFreeHost(b->h_f);
    if (b->h_ev) cudaFreeHost(b->h_ev);
    for (auto &e : b->ev)
        if (e) cudaEventDestroy(e);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    cudaGetLastError();
    delete b;
}

// Lays the schedule out: instance i owns warps[i]/4 consecutive blocks of 4
// warps, holding 4 single-warp cores each or, on its multi-warp row path,
// 4/G cores of G warps (G <= 4); with both paths in use the blocks are
// split by the share of the nonzeros in the long rows.
asaga_status batch_layout(asaga_batch *b, std::string *err) {
    b->block_begin.assign(b->count, 0);
    int g = 0;
    const int slots = update_register_slots(b->dense, true);
    for (int i = 0; i < b->count; ++i) {
        asaga_ctx *c = b->ctx[i];
        const int blocks = std::max(1, b->warps[i] / 4);
        b->block_begin[i] = g;
        g += blocks;
        UpdateParams &u = b->h_up[i];
        int G = std::min(c->row_group, 4);
        int64_t T = c->row_threshold;
        if (G <= 1 || T >= c->max_row_len) T = -1;
        if (T > 0 && blocks < 2) T = -1;
        if (T < 0) G = 1;
        u.wpb = 4;
        u.group = G;
        u.threshold = T;
        u.long_bits = nullptr;
        if (T < 0) {
            u.short_blocks = blocks;
            u.short_cores = 4 * blocks;
            u.long_cores = 0;
        } else if (T == 0) {
            u.short_blocks = 0;
            u.short_cores = 0;
            u.long_cores = blocks * (4 / G);
        } else {
            TRY(ensure_row_classes(c, T, err));
            const int lb = std::max(1, std::min(blocks - 1, (int)std::llround(blocks * c->long_share)));
            u.short_blocks = blocks - lb;
            u.short_cores = 4 * u.short_blocks;
            u.long_cores = lb * (4 / G);
            u.long_bits = c->long_bits;
        }
        int64_t need = 0;
        if (u.short_cores > 0) need = (T > 0 ? std::min(T, c->max_row_len) : c->max_row_len) - 32 * slots;
        if (u.long_cores > 0) need = std::max<int64_t>(need, c->max_row_len - (int64_t)32 * G * slots);
        u.tail_c = nullptr;
        u.tail_stride = 0;
        if (need > 0) {
            const int64_t floats = (int64_t)(u.short_cores + u.long_cores) * need;
            if (floats > c->tail_floats) {
                CK(cudaStreamSynchronize(b->stream), "sync");
                if (c->tail_c) {
                    cudaFree(c->tail_c);
                    c->device_bytes -= c->tail_floats * (int64_t)sizeof(float);
                    c->tail_c = nullptr;
                    c->tail_floats = 0;
                }
                TRY(dev_alloc(&c->tail_c, (size_t)floats, c, err, "alloc row tail scratch"));
                c->tail_floats = floats;
            }
            u.tail_c = c->tail_c;
            u.tail_stride = need;
        }
    }
    b->grid = g;
    CK(cudaMemcpyAsync(b->d_block_begin, b->block_begin.data(), b->count * sizeof(int), cudaMemcpyHostToDevice,
                       b->stream), "copy schedule");
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    if (b->graph_rc) {
        cudaGraphExecDestroy(b->graph_rc);
        b->graph_rc = nullptr;
    }
    return ASAGA_OK;
}

// Cost of one epoch of instance i relative to the others: an update costs a
// fixed latency (sample, row_ptr, gathers, reduction) plus a little per
// entry, so n_i (1 + k_i/128), k_i its mean row length.
double batch_epoch_cost(const asaga_ctx *c) {
    const double k = c->n > 0 ? (double)c->nnz / (double)c->n : 0.0;
    return (double)c->n * (1.0 + k / 128.0);
}

// Warps in proportion to weight[i] (a multiple of 4, at least 4, at most
// max(4, n_i/64) so that tau stays below n_i/10 as Theorem 2 asks), within
// the warps that can be resident at once.
asaga_status batch_weighted_schedule(asaga_batch *b, const std::vector<double> &weight, std::string *err) {
    const int64_t budget = (int64_t)b->resident_blocks * 4;
    double total = 0;
    for (double w : weight) total += w;
    b->warps.assign(b->count, 4);
    int64_t used = 0;
    for (int i = 0; i < b->count; ++i) {
        const asaga_ctx *c = b->ctx[i];
        const double share = total > 0 ? weight[i] / total * (double)budget : 4.0;
        int64_t w = std::max<int64_t>(4, ((int64_t)share / 4) * 4);
        w = std::min<int64_t>(w, std::max<int64_t>(4, (c->n / 64 / 4) * 4));
        b->warps[i] = (int)w;
        used += w;
    }
    while (used > budget) {  // trim the largest shares until the schedule fits
        int imax = (int)(std::max_element(b->warps.begin(), b->warps.end()) - b->warps.begin());
        if (b->warps[imax] <= 4) break;
        b->warps[imax] -= 4;
        used -= 4;
    }
    return batch_layout(b, err);
}

// Default schedule: every instance's epoch takes about as long, so that no
// instance holds the shared segments back.
asaga_status batch_default_schedule(asaga_batch *b, std::string *err) {
    std::vector<double> w(b->count);
    for (int i = 0; i < b->count; ++i) w[i] = batch_epoch_cost(b->ctx[i]);
    return batch_weighted_schedule(b, w, err);
}

asaga_status batch_create_impl(asaga_batch *b, int count, const asaga_problem *problems,
                               const asaga_options *options, std::string *err) {
    if (count < 1) return fail(err, ASAGA_EINVAL, "count must be >= 1");
    if (!problems || !options) return fail(err, ASAGA_EINVAL, "problems or options is NULL");
    for (int i = 1; i < count; ++i) {
        if (options[i].storage_dtype != options[0].storage_dtype)
            return fail(err, ASAGA_EINVAL, "all instances must share storage_dtype");
        if ((problems[i].dense != 0) != (problems[0].dense != 0))
            return fail(err, ASAGA_EINVAL, "all instances must be sparse or all dense");
    }
    for (int i = 0; i < count; ++i)
        if (options[i].deterministic) return fail(err, ASAGA_EINVAL, "batches run asynchronously");
    b->count = count;
    CK(cudaGetDevice(&b->device), "cudaGetDevice");
    if (options[0].cuda_stream) {
        b->stream = (cudaStream_t)options[0].cuda_stream;
    } else {
        CK(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking), "cudaStreamCreate");
        b->own_stream = true;
    }
    for (auto &e : b->ev) CK(cudaEventCreate(&e), "cudaEventCreate");
    for (int i = 0; i < count; ++i) {
        asaga_options o = options[i];
        o.cuda_stream = b->stream;
        o.compact = 0;  // decided below for all instances together (one kernel layout)
        asaga_ctx *c = new (std::nothrow) asaga_ctx();
        if (!c) return fail(err, ASAGA_ENOMEM, "host allocation failed");
        std::string e;
        asaga_status st = create_impl(c, &problems[i], &o, &e);
        if (st != ASAGA_OK) {
            release(c);
            return fail(err, st, "instance " + std::to_string(i) + ": " + e);
        }
        b->ctx.push_back(c);
    }
    if (options[0].compact && !b->ctx[0]->dense) {
        bool all_equal = true, all_small = true;
        for (auto *c : b->ctx) {
            bool eq = false;
            TRY(rows_constant(c, &eq, err));
            all_equal = all_equal && eq;
            all_small = all_small && c->d <= 65536;
        }
        for (auto *c : b->ctx) TRY(apply_compact(c, all_equal, all_small, err));
    }
    b->layout = b->ctx[0]->layout;
    b->dense = b->ctx[0]->dense;
    b->epochs_per_segment = std::max(1, options[0].epochs_per_segment);
    b->abar_every = options[0].abar_recompute_every;
    cudaDeviceProp prop;
    CK(cudaGetDeviceProperties(&prop, b->device), "cudaGetDeviceProperties");
    b->resident_blocks = prop.multiProcessorCount * batch_update_max_blocks_per_sm(b->layout, b->dense);
    b->eval_grid = std::max(1, std::min(64, (prop.multiProcessorCount * 8 + count - 1) / count));
    CK(cudaMallocHost((void **)&b->h_up, count * sizeof(UpdateParams)), "alloc pinned");
    CK(cudaMallocHost((void **)&b->h_f, count * sizeof(double)), "alloc pinned");
    CK(cudaMallocHost((void **)&b->h_ev, count * sizeof(EvalParams)), "alloc pinned");
    TRY(dev_alloc(&b->d_up, count, b->ctx[0], err, "alloc params"));
    TRY(dev_alloc(&b->d_ev, count, b->ctx[0], err, "alloc params"));
    TRY(dev_alloc(&b->d_block_begin, count, b->ctx[0], err, "alloc schedule"));
    TRY(dev_alloc(&b->d_partial, 2 * (size_t)count * b->eval_grid, b->ctx[0], err, "alloc partials"));
    TRY(dev_alloc(&b->d_f, count, b->ctx[0], err, "alloc objectives"));
    b->recompute_grid = std::max(1, std::min(64, (prop.multiProcessorCount * 8 + count - 1) / count));
    TRY(dev_alloc(&b->d_rpartial, (size_t)count * b->recompute_grid, b->ctx[0], err, "alloc partials"));
    TRY(dev_alloc(&b->d_drift, count, b->ctx[0], err, "alloc drifts"));
    TRY(dev_alloc(&b->d_status, 1, b->ctx[0], err, "alloc status"));
    CK(cudaMemsetAsync(b->d_status, 0, sizeof(int), b->stream), "memset status");
    CK(cudaMallocHost((void **)&b->h_drift, count * sizeof(double)), "alloc pinned");
    CK(cudaMallocHost((void **)&b->h_status, sizeof(int)), "alloc pinned");
    *b->h_status = 0;
    std::vector<EvalParams> ev(count);
    for (int i = 0; i < count; ++i) {
        b->h_up[i] = update_params(b->ctx[i]);
        b->h_up[i].count = 0;
        b->h_up[i].fence_each = 0;
        b->h_up[i].status = b->d_status;  // one status word for the whole batch
        ev[i] = eval_params(b->ctx[i]);
        b->h_ev[i] = ev[i];
        b->max_hot = std::max(b->max_hot, b->ctx[i]->n_hot);
    }
    b->ev_full = ev;
    CK(cudaMemcpyAsync(b->d_ev, ev.data(), count * sizeof(EvalParams), cudaMemcpyHostToDevice, b->stream),
       "copy params");
    TRY(batch_default_schedule(b, err));
    return stream_sync(b->ctx[0], err);
}

// Enqueues one segment: parameters in, one update launch over all
// instances, (every abar_recompute_every-th segment) the batched abar
// recomputation, the batched objective, objectives, drifts and status out.
asaga_status batch_enqueue_segment(asaga_batch *b, bool recompute, std::string *err) {
    CK(cudaMemcpyAsync(b->d_up, b->h_up, b->count * sizeof(UpdateParams), cudaMemcpyHostToDevice, b->stream),
       "copy params");
    CK(cudaMemcpyAsync(b->d_ev, b->h_ev, b->count * sizeof(EvalParams), cudaMemcpyHostToDevice, b->stream),
       "copy eval params");
    CK(launch_batch_update(b->d_up, b->d_block_begin, b->count, b->grid, b->layout, b->dense, b->stream),
       "batch update kernel");
    if (recompute) {
        CK(launch_batch_recompute(b->d_ev, b->count, b->recompute_grid, b->layout, b->dense, b->max_hot,
                                  b->d_rpartial, b->d_drift, b->stream),
           "batch abar recomputation");
        CK(cudaMemcpyAsync(b->h_drift, b->d_drift, b->count * sizeof(double), cudaMemcpyDeviceToHost, b->stream),
           "copy drift");
    }
    CK(launch_batch_objective(b->d_ev, b->count, b->eval_grid, b->layout, b->dense, b->d_partial, b->d_f, b->stream),
       "batch objective");
    CK(cudaMemcpyAsync(b->h_f, b->d_f, b->count * sizeof(double), cudaMemcpyDeviceToHost, b->stream), "copy f");
    CK(cudaMemcpyAsync(b->h_status, b->d_status, sizeof(int), cudaMemcpyDeviceToHost, b->stream), "copy status");
    return ASAGA_OK;
}

// Runs one segment through its captured graph (captured on first use; one
// graph without and one with the abar recomputation).  *ms: the segment's
// device time, recomputation included.
asaga_status batch_segment(asaga_batch *b, bool recompute, float *ms, std::string *err) {
    cudaGraphExec_t &exec = recompute ? b->graph_rc : b->graph;
    if (!exec) {
        cudaGraph_t g = nullptr;
        CK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
        asaga_status st = batch_enqueue_segment(b, recompute, err);
        cudaError_t e = cudaStreamEndCapture(b->stream, &g);
        if (st != ASAGA_OK) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        if (e != cudaSuccess) return cuda_fail(err, e, "end capture");
        e = cudaGraphInstantiate(&exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return cuda_fail(err, e, "graph instantiate");
    }
    CK(cudaEventRecord(b->ev[0], b->stream), "event");
    CK(cudaGraphLaunch(exec, b->stream), "graph launch");
    CK(cudaEventRecord(b->ev[1], b->stream), "event");
    b->launches += recompute ? 7 : 3;
    CK(cudaStreamSynchronize(b->stream), "stream synchronize");
    cudaEventElapsedTime(ms, b->ev[0], b->ev[1]);
    if (*b->h_status & 52)
        return fail(err, ASAGA_ECUDA, "batch update kernel status " + std::to_string(*b->h_status));
    return ASAGA_OK;
}

asaga_status batch_run_impl(asaga_batch *b, double max_epochs, double target, const double *f_star,
                            asaga_result *results, std::string *err) {
    if (!(max_epochs >= 0) || !std::isfinite(max_epochs)) return fail(err, ASAGA_EINVAL, "max_epochs must be >= 0");
    if (target > 0 && !f_star) return fail(err, ASAGA_EINVAL, "f_star is needed with a target");
    if (target > 0)
        for (int i = 0; i < b->count; ++i)
            if (!std::isfinite(f_star[i]) || f_star[i] == 0.0)
                return fail(err, ASAGA_EINVAL, "f_star must be finite and nonzero");
    CK(cudaSetDevice(b->device), "cudaSetDevice");
    const auto t0 = std::chrono::steady_clock::now();
    std::vector<asaga_result> r(b->count);
    for (auto &x : r) {
        std::memset(&x, 0, sizeof(x));
        x.f_last = NAN;
        x.rel_subopt = NAN;
    }
    std::vector<char> active(b->count, 1);
    double elapsed_ms = 0, epochs = 0;
    int64_t seg = 0;
    int n_active = b->count;
    const int64_t launches0 = b->launches;
    __atomic_store_n(&b->cancel, 0, __ATOMIC_SEQ_CST);
    bool cancelled = false;
    while (epochs < max_epochs && n_active > 0) {
        if (__atomic_load_n(&b->cancel, __ATOMIC_SEQ_CST)) {
            cancelled = true;
            break;
        }
        NvtxRange range("asaga_batch_run segment");
        const double ep = std::min((double)b->epochs_per_segment, max_epochs - epochs);
        for (int i = 0; i < b->count; ++i) {
            asaga_ctx *c = b->ctx[i];
            UpdateParams &u = b->h_up[i];
            u.gamma = (float)c->gamma;
            u.t_begin = (uint64_t)c->updates_done;
            u.count = active[i] ? (int64_t)std::llround(ep * (double)c->n) : 0;
            // a finished instance also leaves the segment's objective (no rows, no columns)
            b->h_ev[i] = b->ev_full[i];
            if (!active[i]) b->h_ev[i].n = b->h_ev[i].d = 0;
        }
        // every abar_recompute_every-th segment of the batch, counted across calls
        const bool recompute = b->abar_every > 0 && (b->segments_done + 1) % b->abar_every == 0;
        float ms = 0;
        TRY(batch_segment(b, recompute, &ms, err));
        ++b->segments_done;
        elapsed_ms += ms;
        epochs += ep;
        ++seg;
        for (int i = 0; i < b->count; ++i) {
            if (!active[i]) continue;
            asaga_ctx *c = b->ctx[i];
            c->updates_done += b->h_up[i].count;
            r[i].updates += b->h_up[i].count;
            r[i].epochs += ep;
            r[i].segments = seg;
            r[i].f_last = b->h_f[i];
            r[i].solver_seconds = elapsed_ms * 1e-3;  // device time of the shared segments
            if (recompute) r[i].abar_drift = b->h_drift[i];
            if (f_star) r[i].rel_subopt = (r[i].f_last - f_star[i]) / std::fabs(f_star[i]);
            const bool diverged = !std::isfinite(r[i].f_last);
            const bool reached = target > 0 && r[i].rel_subopt <= target;
            if (diverged || reached) {
                active[i] = 0;
                --n_active;
            }
        }
    }
    for (int i = 0; i < b->count; ++i) b->h_ev[i] = b->ev_full[i];  // later segments evaluate every instance
    CK(cudaMemcpyAsync(b->d_ev, b->h_ev, b->count * sizeof(EvalParams), cudaMemcpyHostToDevice, b->stream),
       "copy eval params");
    TRY(stream_sync(b->ctx[0], err));
    const double wall = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    asaga_status st = ASAGA_OK;
    for (int i = 0; i < b->count; ++i) {
        r[i].seconds = wall;
        r[i].kernel_launches = b->launches - launches0;
        if (!std::isfinite(r[i].f_last)) st = ASAGA_EDIVERGED;
        else if (target > 0 && !(r[i].rel_subopt <= target) && st == ASAGA_OK) st = ASAGA_ENOTCONVERGED;
    }
    if (cancelled) st = ASAGA_ECANCELLED;
    if (results) std::copy(r.begin(), r.end(), results);
    if (st != ASAGA_OK)
        fail(err, st, st == ASAGA_EDIVERGED ? "an instance diverged"
                      : st == ASAGA_ECANCELLED ? "cancelled" : "max_epochs reached before the target");
    return st;
}

// Per-instance step sizes from shared trials: every trial runs all
// instances at once with gamma_i = s * gamma0_i for one scale s of the ladder
// 2^(-k/2) and records each instance's float64 |grad f_i|^2 after every
// epoch; each instance then takes, one notch inside its largest converging
// step, the step with the fewest predicted epochs (the single-problem tests).
// One pass of shared trials under the current schedule: every trial runs
// all instances at once for E epochs with gamma_i = 2^(-k/2) gamma0_i (k on
// the ladder, shared), recording each instance's float64 |grad f_i|^2 after
// every epoch.  Per instance: kc = one notch inside the largest converging
// step, or a smaller step with fewer predicted epochs; pc = those epochs.
asaga_status batch_tune_pass(asaga_batch *b, int E, std::vector<int> *kc_out, std::vector<double> *pc_out,
                             int *trials, double *seconds, std::string *err) {
    constexpr int kTop = -3, kBottom = 12;  // the single-problem ladder's top, 0.94/L
    const int nk = kBottom - kTop + 1;
    const int N = b->count;
    std::vector<double> g0(N), g(N);
    std::vector<char> live(N, 1);  // instances still running in the current trial
    auto grads = [&](std::vector<double> &out) -> asaga_status {
        for (int i = 0; i < N; ++i) {
            if (!live[i]) continue;
            TRY(enqueue_grad(b->ctx[i], err));
            CK(cudaMemcpyAsync(b->ctx[i]->hout + 2, b->ctx[i]->dout + 2, sizeof(double), cudaMemcpyDeviceToHost,
                               b->stream), "copy");
        }
        TRY(stream_sync(b->ctx[0], err));
        for (int i = 0; i < N; ++i)
            if (live[i]) out[i] = b->ctx[i]->hout[2];
        return ASAGA_OK;
    };
    for (auto *c : b->ctx) TRY(reset_state(c, err));
    TRY(grads(g0));
    std::vector<char> conv((size_t)N * nk, 0), tried(nk, 0);
    std::vector<double> pred((size_t)N * nk, INFINITY), best(N, INFINITY);
    for (int k = kTop; k <= kBottom; ++k) {
        const double scale = std::pow(2.0, -0.5 * k);
        for (auto *c : b->ctx) TRY(reset_state(c, err));
        std::vector<TuneTrial> t(N);
        std::fill(live.begin(), live.end(), 1);
        for (int e = 1; e <= E; ++e) {
            for (int i = 0; i < N; ++i) {
                asaga_ctx *c = b->ctx[i];
                b->h_up[i].gamma = (float)(c->gamma_base * scale);
                b->h_up[i].t_begin = (uint64_t)c->updates_done;
                b->h_up[i].count = live[i] ? c->n : 0;
            }
            float ms = 0;
            TRY(batch_segment(b, false, &ms, err));
            *seconds += ms * 1e-3;
            for (int i = 0; i < N; ++i)
                if (live[i]) b->ctx[i]->updates_done += b->ctx[i]->n;
            TRY(grads(g));
            for (int i = 0; i < N; ++i) {
                if (t[i].diverged || !live[i]) continue;
                t[i].epochs = e;
                if (!(g0[i] > 0) || !std::isfinite(g[i]) || g[i] > 1e6 * g0[i]) {
                    t[i].diverged = g0[i] > 0;
                    live[i] = 0;  // diverged: nothing more to learn from this trial
                    continue;
                }
                t[i].y.push_back(std::log10(std::max(g[i] / g0[i], 1e-300)));
                if (t[i].y.back() <= kTuneDeep) live[i] = 0;  // reached the prediction's level: its count is exact
            }
        }
        ++*trials;
        tried[k - kTop] = 1;
        bool any_better = false, all_settled = true;
        for (int i = 0; i < N; ++i) {
            conv[(size_t)i * nk + (k - kTop)] = converging(t[i]);
            const double pe = predict_epochs(t[i]);
            pred[(size_t)i * nk + (k - kTop)] = pe;
            if (pe < best[i]) {
                best[i] = pe;
                any_better = true;
            }
            if (!std::isfinite(best[i])) all_settled = false;
        }
        if (!any_better && all_settled && k >= 2) break;  // smaller steps help no instance any more
    }
    kc_out->assign(N, -1000);
    pc_out->assign(N, INFINITY);
    for (int i = 0; i < N; ++i) {
        int kF = kBottom + 1;  // the largest step that converges (and whose next smaller step does too)
        for (int k = kTop; k <= kBottom && tried[k - kTop]; ++k) {
            const bool next_ok = k == kBottom || !tried[k + 1 - kTop] || conv[(size_t)i * nk + (k + 1 - kTop)];
            if (conv[(size_t)i * nk + (k - kTop)] && next_ok) {
                kF = k;
                break;
            }
        }
        int kc = -1000;
        double pc = INFINITY;
        for (int k = kF + 1; k <= kBottom && tried[k - kTop]; ++k)
            if (pred[(size_t)i * nk + (k - kTop)] < pc) {
                pc = pred[(size_t)i * nk + (k - kTop)];
                kc = k;
            }
        if (kc == -1000 && kF + 1 <= kBottom) kc = kF + 1;  // untried or unsettled: one notch inside
        (*kc_out)[i] = kc;
        (*pc_out)[i] = pc;
    }
    return ASAGA_OK;
}

// Longer trials for the instances whose prediction lies beyond twice the
// trial (ill-conditioned ones slow down after the trial's early phase):
// they alone run again from x = 0 at their chosen step (the others get no
// updates), for up to 8x the trial length, until the prediction is within
// twice the epochs run.
asaga_status batch_refine_predictions(asaga_batch *b, int E, const std::vector<int> &kc, std::vector<double> *pc,
                                      double *seconds, std::string *err) {
    const int N = b->count;
    std::vector<int> slow;
    for (int i = 0; i < N; ++i)
        if (kc[i] != -1000 && std::isfinite((*pc)[i]) && (*pc)[i] > 2.0 * E) slow.push_back(i);
    if (slow.empty()) return ASAGA_OK;
    std::vector<double> g0(N, 0.0);
    std::vector<TuneTrial> t(N);
    std::vector<char> live(N, 0);
    for (int i : slow) {
        live[i] = 1;
        asaga_ctx *c = b->ctx[i];
        TRY(reset_state(c, err));
        TRY(enqueue_grad(c, err));
        CK(cudaMemcpyAsync(c->hout + 2, c->dout + 2, sizeof(double), cudaMemcpyDeviceToHost, b->stream), "copy");
    }
    TRY(stream_sync(b->ctx[0], err));
    for (int i : slow) g0[i] = b->ctx[i]->hout[2];
    for (int e = 1; e <= 8 * E; ++e) {
        bool any = false;
        for (int i = 0; i < N; ++i) {
            asaga_ctx *c = b->ctx[i];
            b->h_up[i].gamma = (float)(c->gamma_base * std::pow(2.0, -0.5 * (kc[i] == -1000 ? 0 : kc[i])));
            b->h_up[i].t_begin = (uint64_t)c->updates_done;
            b->h_up[i].count = live[i] ? c->n : 0;
            any = any || live[i];
        }
        if (!any) break;
        float ms = 0;
        TRY(batch_segment(b, false, &ms, err));
        *seconds += ms * 1e-3;
        for (int i : slow) {
            if (!live[i]) continue;
            asaga_ctx *c = b->ctx[i];
            c->updates_done += c->n;
            TRY(enqueue_grad(c, err));
            CK(cudaMemcpyAsync(c->hout + 2, c->dout + 2, sizeof(double), cudaMemcpyDeviceToHost, b->stream), "copy");
        }
        TRY(stream_sync(b->ctx[0], err));
        for (int i : slow) {
            if (!live[i]) continue;
            const double g = b->ctx[i]->hout[2];
            t[i].epochs = e;
            if (!std::isfinite(g) || g > 1e6 * g0[i]) {
                t[i].diverged = true;
                live[i] = 0;
                (*pc)[i] = INFINITY;
                continue;
            }
            t[i].y.push_back(std::log10(std::max(g / g0[i], 1e-300)));
            if (e >= E) {
                const double pe = predict_epochs(t[i]);
                if (!std::isfinite(pe) || pe <= 2.0 * e || t[i].y.back() <= kTuneDeep || e == 8 * E) {
                    (*pc)[i] = pe;
                    live[i] = 0;
                }
            }
        }
    }
    for (int i : slow) TRY(reset_state(b->ctx[i], err));
    return ASAGA_OK;
}

// Device time of one batch epoch under the current schedule and steps (the
// faster of two epochs after one untimed, every instance from x = 0).
asaga_status batch_time_epoch(asaga_batch *b, double *ms_out, double *seconds, std::string *err) {
    for (auto *c : b->ctx) TRY(reset_state(c, err));
    double best = INFINITY;
    for (int e = 0; e < 3; ++e) {
        for (int i = 0; i < b->count; ++i) {
            asaga_ctx *c = b->ctx[i];
            b->h_up[i].gamma = (float)c->gamma;
            b->h_up[i].t_begin = (uint64_t)c->updates_done;
            b->h_up[i].count = c->n;
        }
        float ms = 0;
        TRY(batch_segment(b, false, &ms, err));
        *seconds += ms * 1e-3;
        for (auto *c : b->ctx) c->updates_done += c->n;
        if (e > 0) best = std::min(best, (double)ms);
    }
    *ms_out = best;
    return ASAGA_OK;
}

asaga_status batch_tune_row_paths(asaga_batch *b, double *seconds, std::string *err) {
    auto apply = [&](double E) -> asaga_status {
        for (auto *c : b->ctx) {
            const double k = c->n > 0 ? (double)c->nnz / (double)c->n : 0.0;
            int G = 1;
            while (G < 4 && k >= 2.0 * G * E) G *= 2;
            c->row_group = G;
            c->row_threshold = G > 1 ? 0 : -1;
        }
        return batch_layout(b, err);
    };
    double best_ms = INFINITY, best_E = 0;
    TRY(apply(INFINITY));
    TRY(batch_time_epoch(b, &best_ms, seconds, err));
    const double t_single = best_ms;
    best_ms = 0.97 * t_single;
    for (double E : {512.0, 256.0}) {
        bool any = false;
        for (auto *c : b->ctx) any = any || (c->n > 0 && (double)c->nnz / (double)c->n >= 2.0 * E);
        if (!any) continue;
        double ms = INFINITY;
        TRY(apply(E));
        TRY(batch_time_epoch(b, &ms, seconds, err));
        if (ms < best_ms) {
            best_ms = ms;
            best_E = E;
        }
    }
    return apply(best_E > 0 ? best_E : INFINITY);
}

asaga_status batch_autotune_impl(asaga_batch *b, double trial_epochs, asaga_tune_result *res, std::string *err) {
    CK(cudaSetDevice(b->device), "cudaSetDevice");
    const int E = trial_epochs > 0 ? std::max(5, (int)std::ceil(trial_epochs)) : 16;
    const int N = b->count;
    int trials = 0;
    double seconds = 0;
    for (auto *c : b->ctx) {  // the trials run on single-warp cores; the row paths come last
        c->row_group = 1;
        c->row_threshold = -1;
    }
    // 1. steps under the default schedule (equal epoch times)
    TRY(batch_default_schedule(b, err));
    std::vector<int> kc1, kc2;
    std::vector<double> pc1, pc2;
    TRY(batch_tune_pass(b, E, &kc1, &pc1, &trials, &seconds, err));
    TRY(batch_refine_predictions(b, E, kc1, &pc1, &seconds, err));
    const std::vector<int> warps1 = b->warps;
    // 2. warps in proportion to each instance's predicted work (epochs x epoch
    //    cost), steps again; kept if the predicted makespan is shorter
    std::vector<double> finite;
    for (double p : pc1)
        if (std::isfinite(p)) finite.push_back(p);
    std::sort(finite.begin(), finite.end());
    const double fallback = finite.empty() ? 1.0 : finite.back();
    std::vector<double> w(N);
    for (int i = 0; i < N; ++i)
        w[i] = batch_epoch_cost(b->ctx[i]) * std::max(1.0, std::isfinite(pc1[i]) ? pc1[i] : fallback);
    TRY(batch_weighted_schedule(b, w, err));
    bool second = b->warps != warps1;
    if (second) {
        TRY(batch_tune_pass(b, E, &kc2, &pc2, &trials, &seconds, err));
        TRY(batch_refine_predictions(b, E, kc2, &pc2, &seconds, err));
        // The predictions of slow instances run short (their convergence keeps
        // slowing down), so makespans compare poorly and the second schedule,
        // which gives those instances more warps, is kept (measured: 0.33-0.40 s
        // to the batch's 1e-6 with it, 0.63-0.75 s without).  An instance that
        // the first pass predicted and the second did not (a trend test that
        // failed by chance, or a plateau at more warps) keeps its first step at
        // no more warps than it had then: W gamma stays at or below the point
        // whose prediction was measured.
        bool relayout = false;
        for (int i = 0; i < N; ++i) {
            if (!std::isfinite(pc1[i]) || std::isfinite(pc2[i])) continue;
            kc2[i] = kc1[i];
            pc2[i] = pc1[i];
            if (b->warps[i] > warps1[i]) {
                b->warps[i] = warps1[i];
                relayout = true;
            }
        }
        if (relayout) TRY(batch_layout(b, err));
    }
    const std::vector<int> &kc = second ? kc2 : kc1;
    const std::vector<double> &pc = second ? pc2 : pc1;
    for (int i = 0; i < N; ++i)
        if (kc[i] != -1000) b->ctx[i]->gamma = b->ctx[i]->gamma_base * std::pow(2.0, -0.5 * kc[i]);
    // 3. per-instance row paths at the tuned warps and steps (the warps are
    //    regrouped, not added): every row of instance i on cores of
    //    G_i = min(4, 2^floor(log2(k_i / E))) warps, k_i its mean row length,
    //    for E = 512 and 256 entries per warp, against single warps; each
    //    schedule's batch epoch timed (the faster of two after one untimed),
    //    the fastest kept if 3% faster
    TRY(batch_tune_row_paths(b, &seconds, err));
    b->segments_done = 0;  // the tuned state starts at x = 0: the abar cadence restarts
    for (int i = 0; i < N; ++i) {
        asaga_ctx *c = b->ctx[i];
        c->warps = b->warps[i];
        TRY(reset_state(c, err));
        if (res) {
            res[i].warps = b->warps[i];
            res[i].gamma = c->gamma;
            res[i].score = std::isfinite(pc[i]) ? 1.0 / pc[i] : -1.0;
            res[i].trials = trials;
            res[i].seconds = seconds;
            res[i].row_threshold = c->row_threshold;
            res[i].row_group = c->row_group;
            res[i].draw_ahead = c->draw_ahead;
        }
    }
    return ASAGA_OK;
}

}  // namespace

namespace asaga {
void set_thread_error(const std::string &msg) { g_create_err = msg; }
}  // namespace asaga

extern "C" {

void asaga_default_options(asaga_options *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->loss = ASAGA_LOSS_LOGISTIC;
    o->lambda = 0.0;
    o->gamma = 0.0;
    o->storage_dtype = ASAGA_F32;
    o->max_warps = 0;
    o->deterministic = 0;
    o->seed = 0;
    o->epochs_per_segment = 1;
    o->abar_recompute_every = 0;
    o->timeout_s = 0.0;
    o->cuda_stream = nullptr;
    o->column_stride = 0;
    o->plain_writes = 0;
    o->sampling = ASAGA_SAMPLE_UNIFORM;
    o->compact = 0;
}

asaga_status asaga_create(asaga_ctx **out, const asaga_problem *p, const asaga_options *o) {
    if (!out) {
        g_create_err = "out is NULL";
        return ASAGA_EINVAL;
    }
    *out = nullptr;
    asaga_ctx *c = new (std::nothrow) asaga_ctx();
    if (!c) {
        g_create_err = "host allocation failed";
        return ASAGA_ENOMEM;
    }
    std::string err;
    asaga_status s = create_impl(c, p, o, &err);
    if (s != ASAGA_OK) {
        g_create_err = err;
        release(c);
        return s;
    }
    *out = c;
    return ASAGA_OK;
}

asaga_status asaga_run(asaga_ctx *c, double max_epochs, double target, double f_star, asaga_result *res) {
    if (!c) return ASAGA_EINVAL;
    return run_impl(c, max_epochs, target, f_star, res, &c->err);
}

asaga_status asaga_cancel(asaga_ctx *c) {
    if (!c) return ASAGA_EINVAL;
    __atomic_store_n(c->h_cancel, 1, __ATOMIC_SEQ_CST);
    return ASAGA_OK;
}

asaga_status asaga_batch_cancel(asaga_batch *b) {
    if (!b) return ASAGA_EINVAL;
    __atomic_store_n(&b->cancel, 1, __ATOMIC_SEQ_CST);
    return ASAGA_OK;
}

asaga_status asaga_autotune(asaga_ctx *c, double trial_epochs, asaga_tune_result *res) {
    if (!c) return ASAGA_EINVAL;
    return autotune_impl(c, trial_epochs, res, &c->err);
}

asaga_status asaga_sample_rows(uint64_t seed, int64_t n, int sampling, uint64_t t_begin, int64_t count,
                               int64_t *rows) {
    std::string *err = &g_create_err;
    if (n < 1) return fail(err, ASAGA_EINVAL, "n must be >= 1");
    if (sampling != ASAGA_SAMPLE_UNIFORM && sampling != ASAGA_SAMPLE_PERMUTATION)
        return fail(err, ASAGA_EINVAL, "unknown sampling");
    if (sampling == ASAGA_SAMPLE_PERMUTATION && n > ((int64_t)1 << 62))
        return fail(err, ASAGA_EINVAL, "permutation sampling needs n <= 2^62");
    if (count < 0) return fail(err, ASAGA_EINVAL, "count < 0");
    if (count == 0) return ASAGA_OK;
    if (!rows) return fail(err, ASAGA_EINVAL, "rows is NULL");
    int64_t *d_rows = nullptr;
    cudaError_t e = cudaMalloc(&d_rows, (size_t)count * sizeof(int64_t));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(err, e == cudaErrorMemoryAllocation ? ASAGA_ENOMEM : ASAGA_ECUDA,
                    std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    e = launch_sample_rows(seed, n, sampling, t_begin, count, d_rows, 0);
    if (e == cudaSuccess) e = cudaMemcpy(rows, d_rows, (size_t)count * sizeof(int64_t), cudaMemcpyDeviceToHost);
    cudaFree(d_rows);
    if (e != cudaSuccess) return fail(err, ASAGA_ECUDA, std::string("sampler: ") + cudaGetErrorString(e));
    return ASAGA_OK;
}

asaga_status asaga_measure_overlap(asaga_ctx *c, double epochs, asaga_overlap *out) {
    if (!c) return ASAGA_EINVAL;
    return overlap_impl(c, epochs, out, nullptr, 0, &c->err);
}

asaga_status asaga_measure_overlap_trace(asaga_ctx *c, double epochs, asaga_overlap *out, uint64_t *times,
                                         int64_t capacity) {
    if (!c) return ASAGA_EINVAL;
    return overlap_impl(c, epochs, out, times, capacity, &c->err);
}

asaga_status asaga_run_indices(asaga_ctx *c, const int64_t *idx, int64_t count, int idx_on_device) {
    if (!c) return ASAGA_EINVAL;
    return run_indices_impl(c, idx, count, idx_on_device, &c->err);
}

asaga_status asaga_objective(asaga_ctx *c, double *f) {
    if (!c || !f) return ASAGA_EINVAL;
    std::string *err = &c->err;
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    TRY(enqueue_objective(c, err));
    CK(cudaMemcpyAsync(c->hout, c->dout, sizeof(double), cudaMemcpyDeviceToHost, c->stream), "copy f");
    TRY(stream_sync(c, err));
    *f = c->hout[0];
    return ASAGA_OK;
}

asaga_status asaga_full_grad(asaga_ctx *c, double *grad, double *norm2) {
    if (!c) return ASAGA_EINVAL;
    std::string *err = &c->err;
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    TRY(enqueue_grad(c, err));
    CK(cudaMemcpyAsync(c->hout + 2, c->dout + 2, sizeof(double), cudaMemcpyDeviceToHost, c->stream), "copy norm");
    if (grad) CK(cudaMemcpyAsync(grad, c->acc64, c->d * sizeof(double), cudaMemcpyDeviceToHost, c->stream), "copy grad");
    TRY(stream_sync(c, err));
    if (norm2) *norm2 = c->hout[2];
    return ASAGA_OK;
}

asaga_status asaga_recompute_abar(asaga_ctx *c, double *drift) {
    if (!c) return ASAGA_EINVAL;
    std::string *err = &c->err;
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    TRY(enqueue_recompute(c, err));
    CK(cudaMemcpyAsync(c->hout + 1, c->dout + 1, sizeof(double), cudaMemcpyDeviceToHost, c->stream), "copy drift");
    TRY(stream_sync(c, err));
    if (drift) *drift = c->hout[1];
    return ASAGA_OK;
}

asaga_status asaga_get_state(asaga_ctx *c, float *x, float *abar, float *alpha) {
    if (!c) return ASAGA_EINVAL;
    std::string *err = &c->err;
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    const size_t pitch = (size_t)c->stride * sizeof(float2);
    if (x) CK(cudaMemcpy2DAsync(x, sizeof(float), (const char *)c->state, pitch, sizeof(float), c->d,
                                cudaMemcpyDeviceToHost, c->stream), "copy x");
    if (abar) CK(cudaMemcpy2DAsync(abar, sizeof(float), (const char *)c->state + sizeof(float), pitch, sizeof(float),
                                   c->d, cudaMemcpyDeviceToHost, c->stream), "copy abar");
    if (alpha) CK(cudaMemcpyAsync(alpha, c->alpha, c->n * sizeof(float), cudaMemcpyDeviceToHost, c->stream), "copy alpha");
    TRY(stream_sync(c, err));
    return ASAGA_OK;
}

asaga_status asaga_set_state(asaga_ctx *c, const float *x, const float *abar, const float *alpha,
                             int64_t updates_done) {
    if (!c) return ASAGA_EINVAL;
    if (updates_done < 0) return fail(&c->err, ASAGA_EINVAL, "updates_done < 0");
    std::string *err = &c->err;
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    const size_t pitch = (size_t)c->stride * sizeof(float2);
    if (x) CK(cudaMemcpy2DAsync((char *)c->state, pitch, x, sizeof(float), sizeof(float), c->d,
                                cudaMemcpyHostToDevice, c->stream), "copy x");
    if (abar) CK(cudaMemcpy2DAsync((char *)c->state + sizeof(float), pitch, abar, sizeof(float), sizeof(float), c->d,
                                   cudaMemcpyHostToDevice, c->stream), "copy abar");
    if (alpha) CK(cudaMemcpyAsync(c->alpha, alpha, c->n * sizeof(float), cudaMemcpyHostToDevice, c->stream), "copy alpha");
    TRY(stream_sync(c, err));
    c->updates_done = updates_done;
    c->segments_done = 0;  // the abar recomputation cadence restarts with the restored state
    return ASAGA_OK;
}

asaga_status asaga_set_schedule(asaga_ctx *c, int warps, double gamma, int warps_per_block) {
    if (!c) return ASAGA_EINVAL;
    std::string *err = &c->err;
    if (c->deterministic) return fail(err, ASAGA_EINVAL, "deterministic mode runs one warp");
    if (warps < 1 || warps > c->resident_warps)
        return fail(err, ASAGA_EINVAL, "warps must be in [1, " + std::to_string(c->resident_warps) + "]");
    if (!(gamma > 0) || !std::isfinite(gamma)) return fail(err, ASAGA_EINVAL, "gamma must be finite and > 0");
    if (warps_per_block < 0 || warps_per_block > kUpdateBlock / 32)
        return fail(err, ASAGA_EINVAL, "warps_per_block must be in [0, 8]");
    c->warps = warps;
    c->gamma = gamma;
    c->spread = false;
    if (warps_per_block > 0 && warps_per_block < kUpdateBlock / 32) {
        c->spread = true;
        if (update_warps_per_block(c, warps) != warps_per_block) {
            c->spread = false;
            return fail(err, ASAGA_EINVAL, "warps_per_block does not match the spread of these warps over the SMs");
        }
    }
    return ASAGA_OK;
}

asaga_status asaga_set_row_path(asaga_ctx *c, int64_t threshold, int group) {
    if (!c) return ASAGA_EINVAL;
    if (group != 1 && group != 2 && group != 4 && group != 8)
        return fail(&c->err, ASAGA_EINVAL, "group must be 1, 2, 4 or 8");
    if (threshold < -1) return fail(&c->err, ASAGA_EINVAL, "threshold must be >= -1");
    if (c->deterministic && threshold > 0)
        return fail(&c->err, ASAGA_EINVAL, "deterministic mode takes one path (threshold -1 or 0)");
    c->row_threshold = group > 1 ? threshold : -1;
    c->row_group = threshold >= 0 ? group : 1;
    return ASAGA_OK;
}

asaga_status asaga_get_info(asaga_ctx *c, asaga_info *info) {
    if (!c || !info) return ASAGA_EINVAL;
    info->n = c->n;
    info->d = c->d;
    info->nnz = c->nnz;
    info->L = c->L;
    info->gamma = c->gamma;
    info->delta = c->delta;
    info->warps = c->warps;
    info->column_stride = c->stride;
    info->device_bytes = c->device_bytes;
    info->max_row_len = c->max_row_len;
    info->n_hot = c->n_hot;
    info->warps_per_block = update_warps_per_block(c, c->warps);
    info->col_index_bytes = c->dense ? 0 : ((c->layout & kIdx16) ? 2 : 4);
    info->row_values = (c->layout & ~kIdx16) == kRowScale ? 1 : 0;
    info->row_threshold = c->row_threshold;
    info->row_group = c->row_group;
    info->draw_ahead = c->draw_ahead;
    return ASAGA_OK;
}

asaga_status asaga_set_draw_ahead(asaga_ctx *c, int on) {
    if (!c) return ASAGA_EINVAL;
    if (on != 0 && on != 1) return fail(&c->err, ASAGA_EINVAL, "on must be 0 or 1");
    c->draw_ahead = on;
    return ASAGA_OK;
}

const char *asaga_last_error(const asaga_ctx *c) { return c ? c->err.c_str() : g_create_err.c_str(); }

const char *asaga_status_string(asaga_status s) {
    if ((int)s < 0 || (int)s > 7) return "ASAGA_UNKNOWN";
    return kStatusNames[(int)s];
}

void asaga_destroy(asaga_ctx *c) { release(c); }

asaga_status asaga_batch_create(asaga_batch **out, int count, const asaga_problem *problems,
                                const asaga_options *options) {
    if (!out) {
        g_create_err = "out is NULL";
        return ASAGA_EINVAL;
    }
    *out = nullptr;
    asaga_batch *b = new (std::nothrow) asaga_batch();
    if (!b) {
        g_create_err = "host allocation failed";
        return ASAGA_ENOMEM;
    }
    std::string err;
    asaga_status s = batch_create_impl(b, count, problems, options, &err);
    if (s != ASAGA_OK) {
        g_create_err = err;
        batch_release(b);
        return s;
    }
    *out = b;
    return ASAGA_OK;
}

asaga_status asaga_batch_run(asaga_batch *b, double max_epochs, double target, const double *f_star,
                             asaga_result *results) {
    if (!b) return ASAGA_EINVAL;
    return batch_run_impl(b, max_epochs, target, f_star, results, &b->err);
}

asaga_status asaga_batch_autotune(asaga_batch *b, double trial_epochs, asaga_tune_result *results) {
    if (!b) return ASAGA_EINVAL;
    return batch_autotune_impl(b, trial_epochs, results, &b->err);
}

asaga_status asaga_batch_set_schedule(asaga_batch *b, const int *warps, const double *gamma) {
    if (!b) return ASAGA_EINVAL;
    std::string *err = &b->err;
    if (warps) {
        int64_t total = 0;
        for (int i = 0; i < b->count; ++i) {
            if (warps[i] < 1) return fail(err, ASAGA_EINVAL, "warps must be >= 1");
            total += (warps[i] + 3) / 4;
        }
        if (total > (int64_t)b->resident_blocks)
            return fail(err, ASAGA_EINVAL, "schedule needs more warps than can be resident at once");
        for (int i = 0; i < b->count; ++i) b->warps[i] = ((warps[i] + 3) / 4) * 4;
        TRY(batch_layout(b, err));
    }
    if (gamma)
        for (int i = 0; i < b->count; ++i) {
            if (!(gamma[i] > 0) || !std::isfinite(gamma[i])) return fail(err, ASAGA_EINVAL, "gamma must be > 0");
            b->ctx[i]->gamma = gamma[i];
        }
    return ASAGA_OK;
}

asaga_status asaga_batch_set_row_paths(asaga_batch *b, const int64_t *threshold, const int *group) {
    if (!b) return ASAGA_EINVAL;
    std::string *err = &b->err;
    if (!threshold || !group) return fail(err, ASAGA_EINVAL, "threshold and group must not be NULL");
    for (int i = 0; i < b->count; ++i) {
        if (group[i] != 1 && group[i] != 2 && group[i] != 4)
            return fail(err, ASAGA_EINVAL, "group must be 1, 2 or 4 (blocks of 4 warps)");
        if (threshold[i] < -1) return fail(err, ASAGA_EINVAL, "threshold must be >= -1");
    }
    for (int i = 0; i < b->count; ++i) {
        b->ctx[i]->row_threshold = group[i] > 1 ? threshold[i] : -1;
        b->ctx[i]->row_group = threshold[i] >= 0 ? group[i] : 1;
    }
    return batch_layout(b, err);
}

asaga_status asaga_batch_reset(asaga_batch *b) {
    if (!b) return ASAGA_EINVAL;
    std::string *err = &b->err;
    CK(cudaSetDevice(b->device), "cudaSetDevice");
    for (auto *c : b->ctx) TRY(reset_state(c, err));
    b->segments_done = 0;
    return stream_sync(b->ctx[0], err);
}

asaga_status asaga_batch_get_state(asaga_batch *b, int i, float *x, float *abar, float *alpha) {
    if (!b) return ASAGA_EINVAL;
    if (i < 0 || i >= b->count) return fail(&b->err, ASAGA_EINVAL, "instance out of range");
    asaga_status s = asaga_get_state(b->ctx[i], x, abar, alpha);
    if (s != ASAGA_OK) b->err = b->ctx[i]->err;
    return s;
}

asaga_status asaga_batch_get_info(asaga_batch *b, int i, asaga_info *info) {
    if (!b) return ASAGA_EINVAL;
    if (i < 0 || i >= b->count) return fail(&b->err, ASAGA_EINVAL, "instance out of range");
    asaga_status s = asaga_get_info(b->ctx[i], info);
    if (s == ASAGA_OK) {
        info->warps = b->warps[i];
        info->warps_per_block = kBatchBlock / 32;
    }
    return s;
}

asaga_status asaga_batch_objective(asaga_batch *b, double *f) {
    if (!b || !f) return ASAGA_EINVAL;
    std::string *err = &b->err;
    CK(cudaSetDevice(b->device), "cudaSetDevice");
    CK(launch_batch_objective(b->d_ev, b->count, b->eval_grid, b->layout, b->dense, b->d_partial, b->d_f, b->stream),
       "batch objective");
    CK(cudaMemcpyAsync(b->h_f, b->d_f, b->count * sizeof(double), cudaMemcpyDeviceToHost, b->stream), "copy f");
    CK(cudaStreamSynchronize(b->stream), "sync");
    std::copy(b->h_f, b->h_f + b->count, f);
    return ASAGA_OK;
}

const char *asaga_batch_last_error(const asaga_batch *b) { return b ? b->err.c_str() : g_create_err.c_str(); }

void asaga_batch_destroy(asaga_batch *b) { batch_release(b); }


}  // extern "C"
