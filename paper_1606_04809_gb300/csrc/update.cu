// The asynchronous Sparse SAGA update kernel (Algorithm 2 of arXiv:1606.04809
// with the projected l2 term of Sec. 4.2).
//
// Each concurrent update runs on a "core" (an ASAGA core of Algorithm 2):
// one warp, or, on the multi-warp row path, a group of G warps of one block.
// Update t of a launch samples its row i = sample_row(seed, t) before
// reading anything (Algorithm 2 samples, then reads), reads x^, abar and D
// on S_i and the memory alpha^_i inconsistently (other cores keep adding to
// them), forms
//     delta = phi'_i(a_i.x^) - alpha^_i,
// and adds, atomically at L2,
//     x_v    += -gamma (delta a_iv + D_v (abar_v + lambda x^_v)),
//     abar_v += delta a_iv / n              for v in S_i,
//     alpha_i += delta                      (Algorithm 2 increments alpha_i by delta-alpha).
// Because alpha_i and abar receive exactly matching increments,
// abar = (1/n) sum_i alpha_i a_i holds in exact arithmetic under any
// interleaving of cores.
//
// One read per entry.  Every entry's state {x^_v, abar_v} and D_v is read
// once, before any write of the update; the dot product uses x^_v and the
// scatter uses the term c_v = D_v (abar_v + lambda x^_v) computed from that
// same read, kept in a register (or, past the register slots of a very long
// row, in a per-core scratch array), so the lambda term sees the x^ of the
// dot product, as Sec. 4.2 reads it.
//
// Row paths.  Lane l of warp w of a G-warp core owns the entries
// 32 (q G + w) + l, q = 0, 1, ...; the warps' partial dot products meet in
// shared memory behind one named barrier per update, and every warp then
// scatters its own entries with the same delta.  Rows longer than a
// threshold take the multi-warp path, the others single-warp cores; each
// path's cores take the updates t of the launch whose rows belong to it
// (strided by core), so every update is applied exactly once.
//
// Staging.  A row's CSR data does not depend on the solver state, so each
// core requests it ahead of time: lane 0 of the core's first warp copies the
// row_ptr entries and label of the row four updates ahead (cp.async), and
// the first 256 G column indices and values of the row two updates ahead
// with one bulk copy per array (cp.async.bulk, the Blackwell copy engine),
// completed on a per-stage mbarrier that every warp of the core waits on
// (bounded waits).  The window between reading x^ and writing x, which sets
// the overlap tau, then holds no staging work.
//
// Layout: A in CSR (int64 row_ptr, int32 or uint16 col_idx, values in
// fp32/bf16/fp16 or one value per row) or dense row-major; per-column state
// float2 {x, abar}, so one 8-byte L2 read serves x^_v and abar_v and one
// 8-byte vector reduction updates both; D_v, which never changes, comes from
// an array of its own through the L1-cached read-only path.
#include <algorithm>

#include "asaga_internal.h"
#include "device_common.cuh"

namespace asaga {

constexpr int kSlots = 8;             // register slots per lane: the staged entries of a row
constexpr int kStages = 4;            // staged CSR slices per core (ring)
constexpr int kMetaRing = 8;          // staged row_ptr / label entries per core (ring)
constexpr int kStageEntries = 32 * kSlots;  // entries of a row staged per warp of the core
constexpr uint64_t kStageWaitNs = 200000000ull;  // a staging copy not done after 200 ms is reported

// Header of a staged row, written by the core's producer lane two updates
// ahead and read by all its warps.
struct StageHdr {
    int64_t row;    // sampled row; -1 past the launch's end; -2 malformed range (skipped)
    int64_t start;  // row_ptr[i] (or i d for dense rows)
    int64_t t;      // update index within the launch
    int len;        // entries of the row
    int col_off;    // element offset of the row's first column in the staged column buffer
    int val_off;    // element offset of its first value in the staged value buffer
    int tx;         // bytes the bulk copies deliver (0: nothing to wait for)
    float label, scale;
};

// Per-core control block in shared memory; the staged data follows it.
struct __align__(16) CoreHdr {
    uint64_t mbar[kStages];
    int64_t m_start[kMetaRing];  // row_ptr[i]
    int64_t m_end[kMetaRing];    // row_ptr[i + 1]
    int64_t m_row[kMetaRing];    // i, or -1 past the end
    int64_t m_t[kMetaRing];      // update index of that row
    float m_label[kMetaRing];
    float m_scale[kMetaRing];    // the row's value (RowScale layout)
    StageHdr hdr[kStages];
    float xz[2][kMaxGroup];      // partial dot products of the warps (by update parity)
    float xa[2];                 // alpha^_i read by the first warp
    int xflag[2][kMaxGroup];     // per warp: bit 0 staging copy missing, bit 1 stop requested
};
constexpr int kCoreHdrBytes = (int)((sizeof(CoreHdr) + 127) / 128 * 128);
// staged bytes per array per stage: 256 G entries of <= 4 bytes, plus the
// slack of rounding the copied range out to 16-byte boundaries
__host__ __device__ constexpr int stage_array_bytes(int g) { return kStageEntries * 4 * g + 32; }
__host__ __device__ constexpr int core_ring_bytes(int g) { return kCoreHdrBytes + 2 * kStages * stage_array_bytes(g); }

// (+128: the rings start at the first 128-byte boundary of the dynamic shared memory)
size_t update_smem_bytes(int wpb) { return (size_t)wpb * core_ring_bytes(1) + 128; }

int update_register_slots(bool, bool) { return kSlots; }

// ---------------------------------------------------------------- PTX helpers

__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void red_add_f32(float *p, float v) {
    asm volatile("red.relaxed.gpu.global.add.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
}

__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(smem)), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(smem)), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all_but_newest() {
    asm volatile("cp.async.wait_group 1;" ::: "memory");
}
// Commits every copy this thread has issued and waits for all of them.
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
// One arrival that also announces `tx` bytes of bulk copies to come.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned tx) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(tx)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
    unsigned done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}
// Waits for the phase of `bar` with the given parity to complete; gives up
// (returns false) after kStageWaitNs.  The first test is inline: the copies
// were started two updates earlier and have almost always landed.
__device__ __noinline__ bool mbar_wait_slow(uint64_t *bar, unsigned parity) {
    const uint64_t t0 = globaltimer_ns();
    for (unsigned it = 1;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 15) == 0 && globaltimer_ns() - t0 > kStageWaitNs) return false;
    }
}
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned parity) {
    return mbar_try_wait(bar, parity) || mbar_wait_slow(bar, parity);
}
// Bulk copy of `bytes` (a multiple of 16, both addresses 16-byte aligned)
// from this GPU's global memory into this CTA's shared memory, completing
// on `bar`.  No multicast.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}
__device__ __forceinline__ void core_barrier(int id, int threads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}

// ---------------------------------------------------------------- row data

template <typename T> __device__ __forceinline__ float raw_value(const unsigned char *buf, int k);
template <> __device__ __forceinline__ float raw_value<float>(const unsigned char *buf, int k) {
    return reinterpret_cast<const float *>(buf)[k];
}
template <> __device__ __forceinline__ float raw_value<__nv_bfloat16>(const unsigned char *buf, int k) {
    return __uint_as_float((unsigned)reinterpret_cast<const unsigned short *>(buf)[k] << 16);
}
template <> __device__ __forceinline__ float raw_value<__half>(const unsigned char *buf, int k) {
    return __half2float(__ushort_as_half(reinterpret_cast<const unsigned short *>(buf)[k]));
}
template <typename I> __device__ __forceinline__ int raw_col(const unsigned char *buf, int k) {
    return (int)reinterpret_cast<const I *>(buf)[k];
}

template <typename T> struct ValBytes { static constexpr int value = sizeof(T); };
template <> struct ValBytes<RowScale> { static constexpr int value = 0; };

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

// The updates a core takes, in order (held by the core's first warp).  With
// one path for all rows: t = core, core + cores, ...  With both paths: the
// same candidates, keeping those whose row belongs to this core's path; 32
// candidates are examined at once, one per lane.
struct RowCursor {
    int64_t m = 0;       // next candidate ordinal
    unsigned mask = 0;   // lanes of the current 32 candidates that belong to this path
    int64_t cand_row = -1, cand_t = -1;  // this lane's candidate
    bool done = false;
};

__device__ __forceinline__ int64_t next_row(const UpdateParams &P, RowCursor &c, int core, int ncores, bool want_long,
                                            int lane, bool &bad, int64_t &t_out) {
    if (!P.long_bits) {
        const int64_t t = core + c.m * ncores;
        ++c.m;
        t_out = t;
        return row_of(P, t, bad);
    }
    while (!c.done) {
        if (c.mask == 0) {
            const int64_t t = core + (c.m + lane) * ncores;
            int64_t i = -1;
            bool mine = false;
            if (t < P.count) {
                i = sampled_row(P.sampling, P.seed, P.t_begin + (uint64_t)t, P.n);
                const bool is_long = (__ldg(P.long_bits + (i >> 5)) >> (i & 31)) & 1u;
                mine = is_long == want_long;
            }
            c.mask = __ballot_sync(kFull, mine);
            c.cand_row = i;
            c.cand_t = t;
            c.m += 32;
            if (c.mask == 0 && core + (c.m - 1) * ncores >= P.count) c.done = true;  // the last lane was past the end
            continue;
        }
        const int src = __ffs(c.mask) - 1;
        c.mask &= c.mask - 1;
        t_out = __shfl_sync(kFull, c.cand_t, src);
        return __shfl_sync(kFull, c.cand_row, src);
    }
    t_out = -1;
    return -1;
}

// The core's first warp: lane 0 requests row i's row_ptr entries, label
// (and row value) into meta slot m.
template <typename T, bool kDense>
__device__ __forceinline__ void stage_meta(const UpdateParams &P, CoreHdr &H, int m, int64_t i, int64_t t,
                                           int lane) {
    if (lane != 0) return;
    H.m_row[m] = i;
    H.m_t[m] = t;
    if (i < 0) return;
    if (kDense) {
        H.m_start[m] = i * P.d;
        H.m_end[m] = i * P.d + P.d;
    } else {
        cp_async8(&H.m_start[m], P.row_ptr + i);
        cp_async8(&H.m_end[m], P.row_ptr + i + 1);
    }
    cp_async4(&H.m_label[m], P.labels + i);
    if constexpr (IsRowScale<T>::value) cp_async4(&H.m_scale[m], static_cast<const float *>(P.values) + i);
}

// Lane 0 of the core's first warp, once meta slot m has landed: fills the
// header of stage st and starts the bulk copies of the row's first
// cap = 256 G column indices and values (the copied range rounded out to
// 16-byte boundaries; the allocations of A carry the slack).
template <typename T, typename I, bool kDense>
__device__ __forceinline__ void arm_stage(const UpdateParams &P, CoreHdr &H, unsigned char *data, int m, int st,
                                          int cap, int g) {
    StageHdr &h = H.hdr[st];
    const int64_t i = H.m_row[m];
    h.row = i;
    h.t = H.m_t[m];
    h.tx = 0;
    h.len = 0;
    if (i >= 0) {
        const int64_t start = H.m_start[m], end = H.m_end[m];
        if (start < 0 || end < start || end > P.nnz) {  // a malformed row range: record it, copy nothing
            atomicOr(P.status, 4);
            h.row = -2;
        } else {
            const int len = (int)(end - start);
            const int cnt = len < cap ? len : cap;
            h.start = start;
            h.len = len;
            h.label = H.m_label[m];
            h.scale = IsRowScale<T>::value ? H.m_scale[m] : 0.f;
            unsigned char *colbuf = data + (size_t)st * stage_array_bytes(g);
            unsigned char *valbuf = data + (size_t)(kStages + st) * stage_array_bytes(g);
            unsigned tx = 0;
            const unsigned char *csrc = nullptr, *vsrc = nullptr;
            unsigned cbytes = 0, vbytes = 0;
            if (cnt > 0) {
                if (!kDense) {
                    const int64_t b0 = start * (int64_t)sizeof(I), b1 = (start + cnt) * (int64_t)sizeof(I);
                    const int64_t a0 = b0 & ~(int64_t)15, a1 = (b1 + 15) & ~(int64_t)15;
                    h.col_off = (int)((b0 - a0) / (int64_t)sizeof(I));
                    csrc = static_cast<const unsigned char *>(P.col_idx) + a0;
                    cbytes = (unsigned)(a1 - a0);
                    tx += cbytes;
                }
                if constexpr (!IsRowScale<T>::value) {
                    const int64_t b0 = start * (int64_t)sizeof(T), b1 = (start + cnt) * (int64_t)sizeof(T);
                    const int64_t a0 = b0 & ~(int64_t)15, a1 = (b1 + 15) & ~(int64_t)15;
                    h.val_off = (int)((b0 - a0) / (int64_t)sizeof(T));
                    vsrc = static_cast<const unsigned char *>(P.values) + a0;
                    vbytes = (unsigned)(a1 - a0);
                    tx += vbytes;
                }
            }
            h.tx = (int)tx;
            mbar_arrive_expect_tx(&H.mbar[st], tx);  // release: the header above is visible to the waiters
            if (cbytes) bulk_g2s(colbuf, csrc, cbytes, &H.mbar[st]);
            if (vbytes) bulk_g2s(valbuf, vsrc, vbytes, &H.mbar[st]);
            return;
        }
    }
    mbar_arrive_expect_tx(&H.mbar[st], 0);
}

template <int kN> struct RowRegs {
    int c[kN];      // columns
    float a[kN];    // values
    float cv[kN];   // D_v (abar_v + lambda x^_v) from the update's read of the state
};

// Column and value of entry e from global memory.
template <typename T, typename I, bool kDense>
__device__ __forceinline__ void entry_global(const UpdateParams &P, int64_t start, float scale, int e, int &col,
                                             float &a) {
    col = kDense ? e : col_stream<I>(P.col_idx, start + e);
    if constexpr (IsRowScale<T>::value)
        a = scale;
    else
        a = to_f32(ld_stream(static_cast<const T *>(P.values) + start + e));
}

// One core's share of a launch.  kAhead: the draw placement (P.draw_ahead),
// a template parameter so that the default placement compiles as if the
// option did not exist.
template <typename T, typename I, bool kDense, int kN, bool kAhead>
__device__ __forceinline__ void core_updates(const UpdateParams &P, CoreHdr &H, unsigned char *data, int G, int w,
                                             int lane, int core, int ncores, int core_uid, bool is_long, int bar_id) {
    const int cap = kStageEntries * G;  // staged entries of a row
    const int regcap = 32 * G * kN;     // entries of a row held in registers
    const bool lead = w == 0;           // the core's first warp stages the rows
    float *tail = P.tail_c ? P.tail_c + (int64_t)core_uid * P.tail_stride : nullptr;
    uint64_t deadline = 0;
    if (P.deadline_ns) {  // budget relative to this core's start
        const uint64_t now = __shfl_sync(kFull, globaltimer_ns(), 0);
        deadline = now + P.deadline_ns;
    }
    bool bad = false;
    RowCursor cur;
    int64_t armed = -1;  // last row index (in this core's order) whose stage was armed
    // With P.draw_ahead the first warp draws the row to stage next while the
    // update's gathers are in flight (the sampler's latency is hidden, but
    // the interval between the update's reads and writes grows); otherwise
    // at the top of the update, before its reads.
    constexpr bool draw_ahead = kAhead;
    int64_t next_i = -1, next_t = -1;  // the row drawn ahead (draw_ahead), -1 once the rows ran out
    // prologue: row_ptr entries of rows 0..3, then the slices of rows 0 and 1
    if (lead) {
        int64_t last = -1;
        for (int k = 0; k < 4; ++k) {
            int64_t t;
            const int64_t i = next_row(P, cur, core, ncores, is_long, lane, bad, t);
            stage_meta<T, kDense>(P, H, k, i, t, lane);
            last = i;
        }
        if (draw_ahead && last >= 0) next_i = next_row(P, cur, core, ncores, is_long, lane, bad, next_t);
        if (lane == 0) {
            cp_async_wait_all();
            arm_stage<T, I, kDense>(P, H, data, 0, 0, cap, G);
            arm_stage<T, I, kDense>(P, H, data, 1, 1, cap, G);
        }
        armed = 1;
        __syncwarp();
    }
    if (G > 1) core_barrier(bar_id, 32 * G);
    int64_t k = 0;
    int xb = 0;  // exchanges so far (parity selects the slot)
    bool stop = false;
    for (;; ++k) {
        const int st = (int)(k & (kStages - 1));
        if (lead) {
            // the slice of row k + 2 (its meta was committed two updates ago)
            // and the meta of row k + 4, before this update's reads: the
            // window between its reads and writes then holds no staging work
            // (with draw_ahead, row k + 4 was drawn inside the previous one)
            if (lane == 0) {
                cp_async_wait_all_but_newest();
                arm_stage<T, I, kDense>(P, H, data, (int)((k + 2) & (kMetaRing - 1)), (int)((k + 2) & (kStages - 1)),
                                        cap, G);
            }
            armed = k + 2;
            int64_t i = next_i, t = next_t;
            if constexpr (!draw_ahead) {
                const bool more = H.m_row[(k + 3) & (kMetaRing - 1)] >= 0;
                i = more ? next_row(P, cur, core, ncores, is_long, lane, bad, t) : (t = -1, -1);
            }
            stage_meta<T, kDense>(P, H, (int)((k + 4) & (kMetaRing - 1)), i, t, lane);
            if (lane == 0) cp_async_commit();
            __syncwarp();
        }
        const StageHdr h = H.hdr[st];  // written two updates ago, before a core barrier (or by this warp)
        if (h.row == -1) break;
        const bool live = h.row >= 0;
        bool ok = true;
        if (live && h.tx > 0) ok = mbar_wait_bounded(&H.mbar[st], (unsigned)((k >> 2) & 1));
        ok = __all_sync(kFull, ok);

        // ---- the update's reads (the start of its window)
        RowRegs<kN> r;
        float z = 0.f, alpha_hat = 0.f;
        uint64_t t_read = 0;
        bool scratch_short = false;
        if (live && ok) {
            const unsigned char *colbuf = data + (size_t)st * stage_array_bytes(G);
            const unsigned char *valbuf = data + (size_t)(kStages + st) * stage_array_bytes(G);
            const int len = h.len;
            // the row's data (not the solver state), staged in shared memory
#pragma unroll
            for (int q = 0; q < kN; ++q) {
                const int e = 32 * (q * G + w) + lane;
                r.c[q] = 0;
                r.a[q] = 0.f;
                if (e < len) {
                    r.c[q] = kDense ? e : raw_col<I>(colbuf, h.col_off + e);
                    if constexpr (IsRowScale<T>::value)
                        r.a[q] = h.scale;
                    else
                        r.a[q] = raw_value<T>(valbuf, h.val_off + e);
                }
            }
            if (P.trace && lead) t_read = globaltimer_ns();
            float2 s[kN];
            float dv[kN];
#pragma unroll
            for (int q = 0; q < kN; ++q) {
                s[q] = make_float2(0.f, 0.f);
                dv[q] = 0.f;
                if (32 * (q * G + w) + lane < len) {
                    s[q] = ld_state(P.state + r.c[q] * (int64_t)P.stride);
                    dv[q] = kDense ? 1.f : ld_d(P.dcol + r.c[q]);  // a dense column is in every row: D_v = 1
                }
            }
            if (lead) {
                alpha_hat = __ldcg(P.alpha + h.row);
                if (draw_ahead)  // the row after the one staged above
                    next_i = next_i >= 0 ? next_row(P, cur, core, ncores, is_long, lane, bad, next_t) : -1;
            }
            const float lambda = P.lambda;
#pragma unroll
            for (int q = 0; q < kN; ++q) {
                z = fmaf(r.a[q], s[q].x, z);
                r.cv[q] = dv[q] * fmaf(lambda, s[q].x, s[q].y);
            }
            // entries past the register slots: read once, c_v kept in the scratch
            for (int e = regcap + 32 * w + lane; e < len; e += 32 * G) {
                int cc;
                float av;
                entry_global<T, I, kDense>(P, h.start, h.scale, e, cc, av);
                const float2 sv = ld_state(P.state + cc * (int64_t)P.stride);
                const float dcv = kDense ? 1.f : ld_d(P.dcol + cc);
                z = fmaf(av, sv.x, z);
                const int64_t j = e - regcap;
                if (tail && j < P.tail_stride)
                    tail[j] = dcv * fmaf(lambda, sv.x, sv.y);
                else
                    scratch_short = true;
            }
            z = warp_sum(z);
            alpha_hat = __shfl_sync(kFull, alpha_hat, 0);
        } else if (lead && draw_ahead) {
            next_i = next_i >= 0 ? next_row(P, cur, core, ncores, is_long, lane, bad, next_t) : -1;
        }
        if (__any_sync(kFull, scratch_short)) {
            if (lane == 0) atomicOr(P.status, 32);
            ok = false;
        }
        // stop requests every 32 updates: the deadline, and every 256 the
        // host's cancel flag (a read of mapped host memory)
        int flag = ok ? 0 : 1;
        if ((deadline || P.cancel) && ((k + 1) & 31) == 0 && lead) {
            int s = 0;
            if (lane == 0) {
                if (deadline && globaltimer_ns() > deadline)
                    s = 1;
                else if (P.cancel && ((k + 1) & 255) == 0 && *P.cancel)
                    s = 8;
            }
            s = __shfl_sync(kFull, s, 0);
            if (s) {
                if (lane == 0) atomicOr(P.status, s);
                flag |= 2;
            }
        }
        bool all_ok = ok;
        if (G > 1) {  // partial dot products (and flags) of the core's warps meet here
            const int sl = xb & 1;
            if (lane == 0) {
                H.xz[sl][w] = z;
                H.xflag[sl][w] = flag;
                if (lead) H.xa[sl] = alpha_hat;
            }
            core_barrier(bar_id, 32 * G);
            float zs = 0.f;
            int fl = 0;
            for (int v = 0; v < G; ++v) {  // the same order in every warp
                zs += H.xz[sl][v];
                fl |= H.xflag[sl][v];
            }
            z = zs;
            alpha_hat = H.xa[sl];
            all_ok = (fl & 1) == 0;
            stop = (fl & 2) != 0;
            ++xb;
        } else {
            stop = (flag & 2) != 0;
        }

        // ---- delta and the writes (the end of the window)
        if (live && all_ok) {
            const float delta = phi_prime_f32(P.loss, z, h.label) - alpha_hat;  // the same value in every lane
            const float gamma = P.gamma, inv_n = P.inv_n;
            const int len = h.len;
            if (P.plain_writes) {  // non-thread-safe x_v = x_v + dx (App. G.2 comparison): concurrent adds can be lost
#pragma unroll
                for (int q = 0; q < kN; ++q) {
                    if (32 * (q * G + w) + lane < len) {
                        const float dx = -gamma * fmaf(delta, r.a[q], r.cv[q]);
                        float2 *ptr = P.state + r.c[q] * (int64_t)P.stride;
                        const float2 cur_s = ld_state(ptr);
                        __stcg(ptr, make_float2(cur_s.x + dx, cur_s.y + delta * r.a[q] * inv_n));
                    }
                }
                for (int e = regcap + 32 * w + lane; e < len; e += 32 * G) {
                    int cc;
                    float av;
                    entry_global<T, I, kDense>(P, h.start, h.scale, e, cc, av);
                    const float dx = -gamma * fmaf(delta, av, tail[e - regcap]);
                    float2 *ptr = P.state + cc * (int64_t)P.stride;
                    const float2 cur_s = ld_state(ptr);
                    __stcg(ptr, make_float2(cur_s.x + dx, cur_s.y + delta * av * inv_n));
                }
                if (lead && lane == 0) __stcg(P.alpha + h.row, __ldcg(P.alpha + h.row) + delta);
            } else {
#pragma unroll
                for (int q = 0; q < kN; ++q) {
                    if (32 * (q * G + w) + lane < len) {
                        const float dx = -gamma * fmaf(delta, r.a[q], r.cv[q]);
                        red_add_v2(P.state + r.c[q] * (int64_t)P.stride, dx, delta * r.a[q] * inv_n);
                    }
                }
                for (int e = regcap + 32 * w + lane; e < len; e += 32 * G) {
                    int cc;
                    float av;
                    entry_global<T, I, kDense>(P, h.start, h.scale, e, cc, av);
                    const float dx = -gamma * fmaf(delta, av, tail[e - regcap]);
                    red_add_v2(P.state + cc * (int64_t)P.stride, dx, delta * av * inv_n);
                }
                if (lead && lane == 0) red_add_f32(P.alpha + h.row, delta);
            }
        }
        if (P.trace && lead && lane == 0 && live) {
            P.trace[2 * h.t] = t_read;
            P.trace[2 * h.t + 1] = globaltimer_ns();
        }
        if (P.fence_each) {  // strictly serial order: every write done before the next update reads
            __threadfence();
            __syncwarp();
            if (G > 1) core_barrier(bar_id, 32 * G);
        }
        if (stop || !all_ok) break;
    }
    // no copy may outlive the core's staging area
    if (lead && lane == 0) {
        cp_async_wait_all();
        for (int64_t j = k; j <= armed; ++j) {
            const int sj = (int)(j & (kStages - 1));
            if (!mbar_wait_bounded(&H.mbar[sj], (unsigned)((j >> 2) & 1))) {
                atomicOr(P.status, 16);
                break;
            }
        }
        if (bad) atomicOr(P.status, 2);
    }
    if (lead) __syncwarp();
}

// A block of P.wpb warps: single-warp cores in blocks [0, short_blocks),
// multi-warp cores of P.group warps after.  `block` counts within the
// problem's blocks.
template <typename T, typename I, bool kDense, int kN, bool kAhead>
__device__ __forceinline__ void run_block(const UpdateParams &P, unsigned char *smem, int block) {
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const bool is_long = block >= P.short_blocks;
    const int G = is_long ? P.group : 1;
    const int cpb = P.wpb / G;
    const int cib = wib / G, w = wib - cib * G;
    const int core = (is_long ? block - P.short_blocks : block) * cpb + cib;
    const int ncores = is_long ? P.long_cores : P.short_cores;
    unsigned char *base = smem + ((128 - (smem_addr(smem) & 127)) & 127);  // bulk copies want 16-byte alignment
    unsigned char *ring = base + (size_t)cib * core_ring_bytes(G);
    CoreHdr &H = *reinterpret_cast<CoreHdr *>(ring);
    if (w == 0 && lane == 0) {
        for (int s = 0; s < kStages; ++s) mbar_init(&H.mbar[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    if (wib >= cpb * G || core >= ncores) return;  // whole cores leave together
    const int uid = is_long ? P.short_cores + core : core;
    core_updates<T, I, kDense, kN, kAhead>(P, H, ring + kCoreHdrBytes, G, w, lane, core, ncores, uid, is_long, 1 + cib);
}

template <typename T, typename I, bool kDense, bool kAhead>
__global__ void __launch_bounds__(kUpdateBlock) update_kernel(const UpdateParams P) {
    extern __shared__ __align__(128) unsigned char smem[];
    run_block<T, I, kDense, kSlots, kAhead>(P, smem, (int)blockIdx.x);
}

// Many independent problems in one launch: block b serves instance
// inst = the last i with block_begin[i] <= b, whose parameters are copied to
// shared memory once; its cores split that instance's updates.
template <typename T, typename I, bool kDense>
__global__ void __launch_bounds__(kBatchBlock) batch_update_kernel(const UpdateParams *__restrict__ params,
                                                                   const int *__restrict__ block_begin, int count) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ UpdateParams sp;
    __shared__ int s_first;
    if (threadIdx.x == 0) {
        int lo = 0, hi = count - 1;  // binary search: last instance whose first block <= blockIdx.x
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (block_begin[mid] <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
        }
        s_first = block_begin[lo];
        sp = params[lo];
    }
    __syncthreads();
    if (sp.count <= 0) return;
    run_block<T, I, kDense, kSlots, false>(sp, smem, (int)blockIdx.x - s_first);
}

// Dynamic shared memory beyond 48 KB must be allowed per kernel.
template <typename K> cudaError_t allow_smem(K kernel, size_t bytes) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

struct UpdateLaunch {
    const UpdateParams &p;
    int grid;
    cudaStream_t s;
    template <typename T, typename I, bool kDense, bool kAhead> cudaError_t go() const {
        const size_t smem = update_smem_bytes(p.wpb);
        const cudaError_t e = allow_smem(update_kernel<T, I, kDense, kAhead>, smem);
        if (e != cudaSuccess) return e;
        update_kernel<T, I, kDense, kAhead><<<grid, 32 * p.wpb, smem, s>>>(p);
        return cudaGetLastError();
    }
    template <typename T, typename I, bool kDense> cudaError_t run() const {
        return p.draw_ahead ? go<T, I, kDense, true>() : go<T, I, kDense, false>();
    }
};

cudaError_t launch_update(const UpdateParams &p, int layout, bool dense, int grid, cudaStream_t s) {
    if (p.wpb < 1 || p.wpb * 32 > kUpdateBlock || p.group < 1 || p.group > kMaxGroup || p.wpb % p.group)
        return cudaErrorInvalidValue;
    return with_layout(layout, dense, UpdateLaunch{p, grid, s}, cudaErrorInvalidValue);
}

struct BatchUpdateLaunch {
    const UpdateParams *params;
    const int *block_begin;
    int count, grid;
    cudaStream_t s;
    template <typename T, typename I, bool kDense> cudaError_t run() const {
        const size_t smem = update_smem_bytes(kBatchBlock / 32);
        const cudaError_t e = allow_smem(batch_update_kernel<T, I, kDense>, smem);
        if (e != cudaSuccess) return e;
        batch_update_kernel<T, I, kDense><<<grid, kBatchBlock, smem, s>>>(params, block_begin, count);
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
        cudaError_t e;
        if (batch) {
            const size_t smem = update_smem_bytes(kBatchBlock / 32);
            e = allow_smem(batch_update_kernel<T, I, kDense>, smem);
            if (e == cudaSuccess)
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_update_kernel<T, I, kDense>, kBatchBlock,
                                                                  smem);
        } else {  // the smaller of the two draw placements' figures
            const size_t smem = update_smem_bytes(kUpdateBlock / 32);
            int nb2 = 0;
            e = allow_smem(update_kernel<T, I, kDense, false>, smem);
            if (e == cudaSuccess) e = allow_smem(update_kernel<T, I, kDense, true>, smem);
            if (e == cudaSuccess)
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, update_kernel<T, I, kDense, false>,
                                                                  kUpdateBlock, smem);
            if (e == cudaSuccess)
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb2, update_kernel<T, I, kDense, true>,
                                                                  kUpdateBlock, smem);
            nb = std::min(nb, nb2);
        }
        return e == cudaSuccess && nb > 0 ? nb : 1;
    }
};

int batch_update_max_blocks_per_sm(int layout, bool dense) { return with_layout(layout, dense, UpdateOccupancy{true}, 1); }

int update_max_blocks_per_sm(int layout, bool dense) { return with_layout(layout, dense, UpdateOccupancy{false}, 1); }

// Row classes of the two row paths: bit i of bits <- (row i has more than
// `threshold` entries); sums[0] += entries of those rows, sums[1] += their number.
__global__ void row_classes_kernel(const int64_t *__restrict__ row_ptr, int64_t n, int64_t threshold,
                                   uint32_t *__restrict__ bits, unsigned long long *sums) {
    unsigned long long ent = 0, rows = 0;
    const int64_t words = (n + 31) >> 5;
    for (int64_t wd = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; wd < words;
         wd += (int64_t)gridDim.x * blockDim.x) {
        uint32_t b = 0;
        for (int r = 0; r < 32; ++r) {
            const int64_t i = (wd << 5) + r;
            if (i >= n) break;
            const int64_t len = row_ptr[i + 1] - row_ptr[i];
            if (len > threshold) {
                b |= 1u << r;
                ent += (unsigned long long)len;
                ++rows;
            }
        }
        bits[wd] = b;
    }
    for (int o = 16; o > 0; o >>= 1) {
        ent += __shfl_xor_sync(kFull, ent, o);
        rows += __shfl_xor_sync(kFull, rows, o);
    }
    if ((threadIdx.x & 31) == 0 && (ent || rows)) {
        atomicAdd(sums, ent);
        atomicAdd(sums + 1, rows);
    }
}

cudaError_t launch_row_classes(const int64_t *row_ptr, int64_t n, int64_t threshold, uint32_t *bits,
                               unsigned long long *sums, cudaStream_t s) {
    const int64_t words = (n + 31) >> 5;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(1024, (words + 255) / 256));
    row_classes_kernel<<<grid, 256, 0, s>>>(row_ptr, n, threshold, bits, sums);
    return cudaGetLastError();
}

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
