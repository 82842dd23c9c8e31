// Leaves of the aggregation (Section 4.5: a raw metric is the sum of the
// measured values of one kind in one context).  A leaf is a run of records
// of at most CAP records in one or more consecutive groups (or in one fine
// bin of a big group); its records are summed per key in shared memory:
//   sort: stable LSD radix sort of the packed records, then a warp-striped
//         segmented reduction of the runs of equal keys;
//   hash: an open-addressing table keyed by the record's key accumulates the
//         sums, then only the distinct keys are ordered (rank by counting for
//         a few, radix sort otherwise); a leaf with too many distinct keys
//         falls back to the sort;
//   dense: a leaf of more than CAP records (one fine bin of a big group, at
//         most one window of 8192 subkeys wide) is summed in dense windows.
// Results go to tmp_key / tmp_val at the leaf's start, in key order, with
// the number of keys in leaf_d -- or, for fused leaves (fuse_emit), straight
// to the buffer's output arrays at the offset that a look-back over the
// leaves before it gives, with the per-stall and UNKNOWN totals summed on
// the way (the work k_emit does otherwise).

#include <algorithm>
#include <type_traits>

#include "hpa_internal.h"

namespace hpa {

template <int THREADS, int CAP, bool HAS_CNT, typename V, bool HASH>
struct LeafCfg {
    // 32-bit counts (or none): packed (count, key) elements, digits up to 9
    // bits; 64-bit values: packed (record index, key) elements sorted the
    // same way, the values gathered by index when the runs are summed
    static constexpr bool PACKED = sizeof(V) == 4;
    static constexpr bool IDX = !PACKED && HAS_CNT;
    using E = std::conditional_t<HAS_CNT, uint64_t, uint32_t>;
    using Sort = std::conditional_t<PACKED || IDX, PackedRadix<THREADS, CAP, E>, BlockRadix<THREADS, CAP, 8, V, HAS_CNT>>;
    static constexpr int EPT = (CAP + THREADS - 1) / THREADS;
    static constexpr size_t SORT_BYTES = sizeof(typename Sort::Smem);
    static constexpr int WD = 8192;                              // dense window (uint64 counters)
    // only leaf kernels that may meet a leaf of more than CAP records (an
    // oversized fine bin) carry the dense path; the small-leaf kernel does not
    static constexpr bool DENSE = CAP > SMALL_LEAF_CAP;
    static constexpr size_t DENSE_BYTES = DENSE ? (size_t)WD * 8 : 0;
    // hash aggregation (packed records): an open-addressing table of TS slots
    // (keys u32, sums u64) for at most DMAX - 1 distinct keys, which are then
    // sorted as (slot << 32 | key) elements
    static constexpr int TSLOG = CAP >= 8192 ? 13 : (CAP >= 4096 ? 12 : 10);
    static constexpr int TS = 1 << TSLOG;
    static constexpr int DMAX = TS / 2;
    using HSort = PackedRadix<THREADS, DMAX, uint64_t>;
    static constexpr size_t HASH_BYTES = (PACKED && HASH) ? (size_t)TS * 12 + sizeof(typename HSort::Smem) : 0;
    static constexpr size_t SMEM_SD = SORT_BYTES > DENSE_BYTES ? SORT_BYTES : DENSE_BYTES;
    static constexpr size_t SMEM_WORK = SMEM_SD > HASH_BYTES ? SMEM_SD : HASH_BYTES;
    // fused leaves (packed records, leaf kernels other than the small-leaf
    // one): per-warp per-stall totals and the UNKNOWN totals follow the work area
    static constexpr bool CAN_FUSE = PACKED && CAP > SMALL_LEAF_CAP;
    static constexpr int ACC_WORDS = (THREADS / 32 + 1) * (int)HPA_MAX_STALL_DEV;
    static constexpr size_t SMEM = CAN_FUSE ? ((SMEM_WORK + 15) & ~(size_t)15) + (size_t)ACC_WORDS * 8 : SMEM_WORK;
};

// Look-back over the leaves of one buffer (fused leaves).  Leaf l publishes
// its key count, adds up the counts of the leaves before it, walking back
// until a leaf whose inclusive prefix is published (the buffer's first leaf
// publishes one at once), and publishes its own inclusive prefix.  Leaves
// are taken in index order from a counter, so every leaf waited for has been
// taken by a running CTA that never waits for a later leaf.
//   try:    waits at most `quick` polls; on success the leaf's prefix is
//           published with LOOK_DIRECT (its keys go straight to the output);
//           otherwise only its count is published, its keys go to tmp_key /
//           tmp_val for k_emit, and `finish` completes the walk afterwards,
//           so that a slow leaf delays the leaves after it by at most `quick`
//           polls instead of holding them all (a convoy);
//   finish: bounded by timeout_iters polls; on a timeout the status becomes
//           HPA_E_TIMEOUT and the prefix is published as if the missing
//           counts were zero, so that no CTA waits forever.

// walk back from leaf l - 1 summing counts until an inclusive prefix; false
// if `limit` polls pass first (the sum so far is then incomplete)
__device__ bool leaf_walk(const AggWork& w, uint32_t l, uint32_t first, uint32_t limit, unsigned long long* prefix) {
    unsigned long long sum = 0;
    uint32_t j = l - 1, polls = 0;
    for (;;) {
        const unsigned long long st = ld_acquire_u64(&w.leaf_look[j]);
        if (st & LOOK_INCL) { sum += st & LOOK_VAL; break; }
        if (st & LOOK_AGG) {
            sum += st & LOOK_VAL;
            if (j == first) break;
            --j;
            continue;
        }
        if (++polls > limit) { *prefix = sum; return false; }
        if (limit > LOOK_QUICK) __nanosleep(64);
    }
    *prefix = sum;
    return true;
}

__device__ bool leaf_lookback_try(const AggWork& w, uint32_t l, uint32_t first, uint32_t cnt,
                                  unsigned long long* base) {
    if (l == first) {
        st_release_u64(&w.leaf_look[l], LOOK_INCL | LOOK_DIRECT | cnt);
        *base = 0;
        return true;
    }
    st_release_u64(&w.leaf_look[l], LOOK_AGG | cnt);
    unsigned long long prefix;
    if (!leaf_walk(w, l, first, LOOK_QUICK, &prefix)) return false;
    st_release_u64(&w.leaf_look[l], LOOK_INCL | LOOK_DIRECT | (prefix + cnt));
    *base = prefix;
    return true;
}

__device__ void leaf_lookback_finish(const AggWork& w, uint32_t l, uint32_t first, uint32_t cnt) {
    unsigned long long prefix;
    if (!leaf_walk(w, l, first, w.timeout_iters ? w.timeout_iters : (1u << 22), &prefix))
        raise_status(w.status, 7 /* HPA_E_TIMEOUT */, 11);
    st_release_u64(&w.leaf_look[l], LOOK_INCL | (prefix + cnt));
}

// Where a fused leaf's keys go: the buffer's output arrays from `base`, the
// context of group-tag 0, UNKNOWN coded as node M, and the subkey layout.
struct LeafOut {
    uint32_t* key_ctx;
    uint32_t* key_node;
    uint8_t* key_stall;
    unsigned long long* val;
    uint64_t capacity;
    uint32_t gctx0, M, sbits, sb;
};

// One key of a fused leaf: its per-stall total (this warp's row of counters)
// and UNKNOWN total, and the four output arrays when it is within capacity.
__device__ __forceinline__ void fused_put(const LeafOut& o, uint64_t base, unsigned long long* acc,
                                          unsigned long long* unk, uint32_t pos, uint32_t k, unsigned long long v) {
    const uint32_t smask = o.sbits >= 32 ? 0xFFFFFFFFu : ((1u << o.sbits) - 1);
    const uint32_t sub = k & smask, node = sub >> o.sb, stall = sub & ((1u << o.sb) - 1);
    atomicAdd(&acc[stall], v);
    if (node == o.M) atomicAdd(&unk[stall], v);
    const uint64_t p = base + pos;
    if (p < o.capacity) {
        const uint32_t gl = o.sbits >= 32 ? 0u : (k >> o.sbits);
        __stcs(&o.key_ctx[p], o.gctx0 + gl);
        __stcs(&o.key_node[p], node == o.M ? UNKNOWN : node);
        o.key_stall[p] = (uint8_t)stall;
        __stcs(&o.val[p], v);
    }
}

// Runs of equal keys in a sorted shared-memory array, reduced warp-striped:
// warp w owns a contiguous chunk and walks it 32 elements per row (lane l
// reads element row * 32 + l, so shared-memory reads are conflict-free).
// Run sums come from a segmented inclusive scan per row plus a carry for the
// run still open at the row's (and the previous warp's) end.

template <typename V, bool HAS_V>
__device__ __forceinline__ unsigned long long val_at(const V* vals, int i) {
    if constexpr (HAS_V) return (unsigned long long)vals[i];
    else return 1ull;
}

// mode 0: write every run at its run id; mode 1: count runs with a non-zero
// sum; mode 2: write only runs with a non-zero sum, compacted from nz_base.
// KA(i) gives the key of element i, VA(i) its value; T is the accumulation
// type (32-bit when the leaf's values cannot overflow it).  A run's partial
// sum in a row is the row's inclusive prefix minus the prefix just before the
// run's head (found with a ballot), so one plain scan serves every run.
// put(write, position, key, sum) is called by every lane of the warp
// together; lanes with `write` store one key.
template <typename T, typename KA, typename VA, typename PUT>
__device__ __forceinline__ uint32_t warp_runs(KA K, VA Vf, int n, int w0, int w1,
                                              int run0, T carry, int mode, uint32_t nz_base, PUT put) {
    const int lane = lane_id();
    int run = run0;
    uint32_t nz = nz_base, nz_count = 0;
    // two rows at a time: their scans are independent, only the carry links them
#pragma unroll 2
    for (int base = w0; base < w1; base += 32) {
        const int i = base + lane;
        const bool ok = i < w1;
        const uint32_t k = ok ? K(i) : 0u;
        // neighbours from the adjacent lanes; the row's edge lanes load theirs
        uint32_t kp = __shfl_up_sync(0xffffffffu, k, 1);
        if (lane == 0 && i > 0) kp = K(i - 1);
        uint32_t kn = __shfl_down_sync(0xffffffffu, k, 1);
        if ((lane == 31 || i + 1 >= w1) && i + 1 < n) kn = K(i + 1);
        const bool h = ok && (i == 0 || kp != k);
        const T v = ok ? (T)Vf(i) : T(0);
        const uint32_t hb = __ballot_sync(0xffffffffu, h);
        T p = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const T t = __shfl_up_sync(0xffffffffu, p, o);
            if (lane >= o) p += t;
        }
        const uint32_t le = hb & (lanemask_lt() | (1u << lane));
        const int hpos = le ? 31 - __clz(le) : 0;
        const T ph = __shfl_sync(0xffffffffu, p, hpos > 0 ? hpos - 1 : 0);
        const T sum = le ? (hpos > 0 ? p - ph : p) : p + carry;
        const int rid = run + __popc(le);
        const bool end = ok && (i == n - 1 || kn != k);
        if (mode == 0) {
            put(end, (uint32_t)rid, k, (unsigned long long)sum);
        } else {
            const uint32_t nzb = __ballot_sync(0xffffffffu, end && sum != 0);
            if (mode == 2) put(end && sum != 0, nz + __popc(nzb & lanemask_lt()), k, (unsigned long long)sum);
            nz += __popc(nzb);
            nz_count += __popc(nzb);
        }
        run += __popc(hb);
        carry = __shfl_sync(0xffffffffu, sum, 31);
    }
    return nz_count;
}

// per-warp heads and the partial sum of the run left open at the chunk's end
template <typename T>
struct RunSum {
    uint32_t heads;
    T tail;
    uint32_t has_head;
};

template <typename T, typename KA, typename VA>
__device__ __forceinline__ RunSum<T> warp_run_summary(KA K, VA Vf, int w0, int w1) {
    const int lane = lane_id();
    RunSum<T> r{0, T(0), 0};
    // two rows at a time: their scans are independent, only the carry links them
#pragma unroll 2
    for (int base = w0; base < w1; base += 32) {
        const int i = base + lane;
        const bool ok = i < w1;
        const uint32_t k = ok ? K(i) : 0u;
        uint32_t kp = __shfl_up_sync(0xffffffffu, k, 1);
        if (lane == 0 && i > 0) kp = K(i - 1);
        const bool h = ok && (i == 0 || kp != k);
        const T v = ok ? (T)Vf(i) : T(0);
        const uint32_t hb = __ballot_sync(0xffffffffu, h);
        r.heads += __popc(hb);
        const int last = hb ? 31 - __clz(hb) : 0;
        T x = lane >= last ? v : T(0);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (hb) { r.tail = x; r.has_head = 1; }
        else r.tail += x;
    }
    return r;
}

// Runs of one leaf: per-warp summaries, a block-level (segmented) scan over
// the warps, then every warp writes its runs; keys with a zero sum are
// dropped by a compacting second walk (only when a zero value exists).
// pre(n_out) is called by every thread once the number of keys is known and
// before any key is written (fused leaves find their output offset there).
// Returns the number of keys written.
template <typename T, int W, typename KA, typename VA, typename PRE, typename PUT>
__device__ uint32_t leaf_runs(KA Kc, VA Vc, int n, int w0, int w1, bool any_zero, PRE pre, PUT put,
                              uint32_t* s_run0, uint32_t* s_nz, T* s_carry, uint32_t* s_tot) {
    const int warp = threadIdx.x >> 5, lane = lane_id();
    const RunSum<T> rc = warp_run_summary<T>(Kc, Vc, w0, w1);
    if (lane == 0) { s_run0[warp] = rc.heads; s_carry[warp] = rc.tail; s_nz[warp] = rc.has_head; }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t runs = 0;
        T open = 0;
        for (int x = 0; x < W; ++x) {
            const uint32_t hcount = s_run0[x], hh = s_nz[x];
            const T t = s_carry[x];
            s_run0[x] = runs;
            s_carry[x] = open;
            runs += hcount;
            open = hh ? t : open + t;
        }
        *s_tot = runs;
    }
    __syncthreads();
    uint32_t n_out = *s_tot;
    const int run0 = (int)s_run0[warp] - 1;
    const T carry = s_carry[warp];
    if (!any_zero) {
        pre(n_out);
        warp_runs<T>(Kc, Vc, n, w0, w1, run0, carry, 0, 0, put);
    } else {
        auto none = [](bool, uint32_t, uint32_t, unsigned long long) {};
        const uint32_t nzc = warp_runs<T>(Kc, Vc, n, w0, w1, run0, carry, 1, 0, none);
        __syncthreads();
        if (lane == 0) s_nz[warp] = nzc;
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t t = 0;
            for (int x = 0; x < W; ++x) { const uint32_t c = s_nz[x]; s_nz[x] = t; t += c; }
            *s_tot = t;
        }
        __syncthreads();
        n_out = *s_tot;
        pre(n_out);
        warp_runs<T>(Kc, Vc, n, w0, w1, run0, carry, 2, s_nz[warp], put);
    }
    __syncthreads();
    return n_out;
}

template <int THREADS, int CAP, bool HAS_CNT, typename V, bool HASH>
__global__ void __launch_bounds__(THREADS, THREADS <= 128 ? 8 : (THREADS <= 256 ? 2 : 1))
k_leaf(AggWork w, uint32_t n_lo, uint32_t n_hi) {
    using Cfg = LeafCfg<THREADS, CAP, HAS_CNT, V, HASH>;
    using Sort = typename Cfg::Sort;
    constexpr int W = THREADS / 32;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    typename Sort::Smem& S = *reinterpret_cast<typename Sort::Smem*>(smem_raw);
    __shared__ uint32_t sw[33];
    __shared__ uint32_t gb[1025];
    __shared__ unsigned long long red[2];
    __shared__ uint32_t s_run0[W], s_nz[W];
    __shared__ unsigned long long s_carry[W];
    __shared__ uint32_t s_any_zero, s_tot;
    __shared__ uint32_t s_hd, s_abort;
    __shared__ unsigned long long s_spec;
    __shared__ uint32_t s_leaf, s_direct;
    __shared__ unsigned long long s_base;
    const uint32_t n_leaves = w.item_nleaf[w.G];
    const uint32_t* seg = w.grp_hist;
    const int warp = threadIdx.x >> 5, lane = lane_id();

    // fused leaves: taken in index order from the ticket counter; per-warp
    // per-stall totals and UNKNOWN totals in shared memory, flushed to the
    // buffer's totals when the CTA moves on to another buffer and at the end
    const bool fuse = Cfg::CAN_FUSE && w.fuse_emit != 0;
    unsigned long long* acc = reinterpret_cast<unsigned long long*>(smem_raw + ((Cfg::SMEM_WORK + 15) & ~(size_t)15));
    unsigned long long* unk = acc + W * HPA_MAX_STALL_DEV;
    uint32_t cur_b = 0xFFFFFFFFu;
    if constexpr (Cfg::CAN_FUSE) {
        if (fuse)
            for (int i = threadIdx.x; i < Cfg::ACC_WORDS; i += THREADS) acc[i] = 0;
    }
    auto flush = [&]() {
        __syncthreads();
        if (cur_b != 0xFFFFFFFFu && w.emit_totals) {
            const BufDev& B = w.bufs[cur_b];
            for (uint32_t r = threadIdx.x; r < HPA_MAX_STALL_DEV; r += THREADS) {
                unsigned long long t = 0;
                for (int x = 0; x < W; ++x) { t += acc[x * HPA_MAX_STALL_DEV + r]; acc[x * HPA_MAX_STALL_DEV + r] = 0; }
                const unsigned long long u = unk[r];
                unk[r] = 0;
                if (t && B.total) atomicAdd((unsigned long long*)&B.total[r], t);
                if (u && B.unknown) atomicAdd((unsigned long long*)&B.unknown[r], u);
            }
        }
        __syncthreads();
    };
    auto next_leaf = [&](uint32_t l) -> uint32_t {
        if (!fuse) return l + gridDim.x;
        __syncthreads();                                   // every thread has read s_leaf
        if (threadIdx.x == 0) s_leaf = atomicAdd(w.leaf_ticket, 1u);
        __syncthreads();
        return s_leaf;
    };

    for (uint32_t l = fuse ? next_leaf(0) : blockIdx.x; l < n_leaves; l = next_leaf(l)) {
        const uint32_t start = w.leaf_start[l], end = w.leaf_end[l];
        const uint32_t info = w.leaf_info[l];
        const uint32_t n = end - start;
        if (n < n_lo || n > n_hi) continue;               // another leaf kernel's size class
        // fused leaves: the buffer's output arrays; keys of a buffer with
        // invalid samples are not written (the call fails as a whole)
        LeafOut lo_{};
        uint32_t first = 0;
        bool skip = true;
        if constexpr (Cfg::CAN_FUSE) {
            if (fuse) {
                const uint32_t b = info >> 8;
                if (b != cur_b) {
                    flush();
                    cur_b = b;
                }
                const BufDev& B = w.bufs[b];
                first = w.buf_first_leaf[b];
                skip = w.buf_bad[b] != 0;
                lo_ = LeafOut{B.key_ctx, B.key_node, B.key_stall, (unsigned long long*)B.val, B.capacity,
                              w.leaf_grp0[l] - B.grp_base, w.bins[B.bin].n_nodes, w.sbits, w.sb};
            }
        }
        // pre: the output offset of this leaf if its predecessors have (nearly)
        // published theirs (thread 0 looks back, every thread waits for it);
        // s_direct says whether the keys go straight to the output
        auto pre = [&](uint32_t n_keys) {
            if constexpr (Cfg::CAN_FUSE) {
                if (fuse) {
                    if (threadIdx.x == 0) {
                        unsigned long long b = 0;
                        s_direct = leaf_lookback_try(w, l, first, n_keys, &b) ? 1u : 0u;
                        s_base = b;
                    }
                    __syncthreads();
                }
            }
        };
        // after the keys are written: a leaf that left them to k_emit completes its look-back
        auto post = [&](uint32_t n_keys) {
            if constexpr (Cfg::CAN_FUSE) {
                if (fuse && !s_direct && threadIdx.x == 0) leaf_lookback_finish(w, l, first, n_keys);
            }
        };
        unsigned long long* acc_w = acc + warp * HPA_MAX_STALL_DEV;
        auto put_fused = [&](bool wr, uint32_t pos, uint32_t k, unsigned long long v) {
            if constexpr (Cfg::CAN_FUSE) {
                if (!wr) return;
                if (s_direct) {
                    if (!skip) fused_put(lo_, s_base, acc_w, unk, pos, k, v);
                } else {
                    w.tmp_key[start + pos] = k;
                    w.tmp_val[start + pos] = v;
                }
            }
        };
        // fused leaves whose path left its keys at tmp_key / tmp_val + start:
        // copied to the output when the offset is ready, else left to k_emit
        auto copy_fused = [&](uint32_t n_keys) {
            __syncthreads();
            pre(n_keys);
            if (s_direct)
                for (uint32_t i = threadIdx.x; i < n_keys; i += THREADS)
                    put_fused(true, i, w.tmp_key[start + i], (unsigned long long)w.tmp_val[start + i]);
            post(n_keys);
        };
        const bool second = info & 1u;
        const uint2* src_pair = second ? w.rec2_pair : w.rec_pair;
        const uint32_t* src_sub = second ? w.rec2_sub : w.rec_sub;
        const uint64_t* src_v64 = second ? w.rec2_v64 : w.rec_v64;
        auto rec = [&](uint32_t i, uint32_t& k, unsigned long long& v) {
            if constexpr (HAS_CNT && sizeof(V) == 4) {
                const uint2 r = src_pair[i];
                k = r.x; v = r.y;
            } else {
                k = src_sub[i];
                if constexpr (HAS_CNT) v = src_v64[i]; else v = 1ull;
            }
        };
        if (n == 0) {
            pre(0);
            post(0);
            if (threadIdx.x == 0) w.leaf_d[l] = 0;
            continue;
        }
        if (n <= (uint32_t)CAP) {
            // groups of this leaf: a sub-bin holds one group; an item holds the
            // groups whose records lie in [start, end)
            const uint32_t g0 = w.leaf_grp0[l];
            uint32_t ng = 1;
            if (!second) {
                uint32_t lo = g0, hi = min(w.G, g0 + 1024u);
                while (hi - lo > 1) {
                    const uint32_t m = (lo + hi) >> 1;
                    if (seg[m] < end) lo = m; else hi = m;
                }
                ng = lo - g0 + 1;
            }
            const uint32_t gbits = ng > 1 ? ceil_log2_u64(ng) : 0;
            if (ng > 1) {
                for (uint32_t j = threadIdx.x; j <= ng; j += THREADS) gb[j] = seg[g0 + j] - start;
                __syncthreads();
            }
            if constexpr (Cfg::PACKED && HASH) {
                // Hash aggregation: records are summed into a shared-memory
                // open-addressing table keyed by their (group-tagged) key, of
                // 2^tlog >= 2n slots (at most Cfg::TS), so a leaf of at most
                // TS / 2 records never fills it past one half; a larger leaf
                // with TS / 2 - 1 or more distinct keys falls back to sorting
                // its records.  Only the distinct keys are then ordered.
                constexpr uint32_t EMPTY = 0xFFFFFFFFu;
                using HS = typename Cfg::HSort;
                const int tlog = min(Cfg::TSLOG, max(5, (int)ceil_log2_u64(2ull * n)));
                const uint32_t ts = 1u << tlog;
                uint32_t* hk = reinterpret_cast<uint32_t*>(smem_raw);
                unsigned long long* hv = reinterpret_cast<unsigned long long*>(smem_raw + (size_t)Cfg::TS * 4);
                typename HS::Smem& HM = *reinterpret_cast<typename HS::Smem*>(smem_raw + (size_t)Cfg::TS * 12);
                for (uint32_t j = threadIdx.x; j < ts; j += THREADS) { hk[j] = EMPTY; hv[j] = 0; }
                if (threadIdx.x == 0) { s_hd = 0; s_abort = 0; s_spec = 0; }
                __syncthreads();
                volatile uint32_t* abort_flag = &s_abort;
                volatile uint32_t* vk = hk;
                for (uint32_t i = threadIdx.x; i < n; i += THREADS) {
                    if (*abort_flag) break;
                    uint32_t k;
                    unsigned long long v;
                    rec(start + i, k, v);
                    if (v == 0) continue;                      // adds nothing; zero-sum keys are omitted
                    if (ng > 1) {                              // group within the leaf: last j with gb[j] <= i
                        uint32_t lo = 0, hi = ng;
                        while (hi - lo > 1) {
                            const uint32_t m = (lo + hi) >> 1;
                            if (gb[m] <= i) lo = m; else hi = m;
                        }
                        k |= lo << w.sbits;
                    }
                    if (k == EMPTY) { atomicAdd(&s_spec, v); continue; }   // the one key equal to EMPTY
                    uint32_t h = (k * 2654435769u) >> (32 - tlog);
                    bool placed = false;
                    for (uint32_t t = 0; t < ts; ++t) {
                        uint32_t cur = vk[h];
                        if (cur == EMPTY) {
                            cur = atomicCAS(&hk[h], EMPTY, k);
                            if (cur == EMPTY) {
                                cur = k;
                                if (atomicAdd(&s_hd, 1u) + 1 >= ts / 2) *abort_flag = 1;
                            }
                        }
                        if (cur == k) { atomicAdd(&hv[h], v); placed = true; break; }
                        h = (h + 1) & (ts - 1);
                    }
                    if (!placed) *abort_flag = 1;
                }
                __syncthreads();
                if (!s_abort) {
                    // occupied slots -> (slot << 32 | key) elements (any order:
                    // the keys are distinct)
                    if (threadIdx.x == 0) s_hd = 0;
                    __syncthreads();
                    for (uint32_t j = threadIdx.x; j < ts; j += THREADS) {
                        const uint32_t k = hk[j];
                        if (k != EMPTY) HM.el[0][atomicAdd(&s_hd, 1u)] = ((uint64_t)j << 32) | k;
                    }
                    __syncthreads();
                    uint32_t D = s_hd;
                    if (s_spec) {
                        if (threadIdx.x == 0) HM.el[0][D] = ((uint64_t)Cfg::TS << 32) | EMPTY;
                        ++D;
                    }
                    __syncthreads();
                    auto put = [&](uint32_t pos, uint64_t e) {
                        const uint32_t slot = (uint32_t)(e >> 32);
                        w.tmp_key[start + pos] = (uint32_t)e;
                        w.tmp_val[start + pos] = slot == (uint32_t)Cfg::TS ? s_spec : hv[slot];
                    };
                    if (D <= (uint32_t)THREADS) {
                        // few distinct keys: each element's rank is the number of smaller keys
                        if (threadIdx.x < D) {
                            const uint64_t e = HM.el[0][threadIdx.x];
                            const uint32_t k = (uint32_t)e;
                            uint32_t r = 0;
                            for (uint32_t j = 0; j < D; ++j) r += (uint32_t)HM.el[0][j] < k;
                            put(r, e);
                        }
                    } else {
                        const int hc = HS::sort(HM, (int)D, (int)(w.sbits + gbits), (int)w.sort_mode, w.status);
                        for (uint32_t j = threadIdx.x; j < D; j += THREADS) put(j, HM.el[hc][j]);
                    }
                    if (fuse) copy_fused(D);
                    if (threadIdx.x == 0) w.leaf_d[l] = D;
                    __syncthreads();
                    continue;
                }
            }
            uint32_t zero = 0;
            unsigned long long vmax = 1;
            if constexpr (Cfg::PACKED) {
                // records land in shared memory verbatim, without a register round trip
                for (uint32_t i = threadIdx.x; i < n; i += THREADS) {
                    if constexpr (HAS_CNT) cp_async8(&S.el[0][i], &src_pair[start + i]);
                    else cp_async4(&S.el[0][i], &src_sub[start + i]);
                }
                cp_async_wait_all();
                if constexpr (HAS_CNT)
                    for (uint32_t i = threadIdx.x; i < n; i += THREADS) {
                        const uint32_t v = Sort::val_of(S.el[0][i]);
                        zero |= v == 0;
                        vmax = max(vmax, (unsigned long long)v);
                    }
            } else if constexpr (Cfg::IDX) {
                for (uint32_t i = threadIdx.x; i < n; i += THREADS) {
                    const unsigned long long v = src_v64[start + i];
                    S.el[0][i] = (uint64_t)src_sub[start + i] | ((uint64_t)i << 32);
                    zero |= v == 0;
                    vmax = max(vmax, v);
                }
            } else {
                for (uint32_t i = threadIdx.x; i < n; i += THREADS) {
                    uint32_t k;
                    unsigned long long v;
                    rec(start + i, k, v);
                    S.key[0][i] = k;
                    if constexpr (HAS_CNT) { S.val[0][i] = (V)v; zero |= v == 0; vmax = max(vmax, v); }
                }
            }
            if (threadIdx.x == 0) s_any_zero = 0;
            __syncthreads();
            if (zero) s_any_zero = 1;
            if (ng > 1) {
                // tag each record with its group inside the leaf
                for (uint32_t j = threadIdx.x; j < ng; j += THREADS) {
                    const uint32_t a = gb[j], e = min(gb[j + 1], n);
                    for (uint32_t i = a; i < e; ++i) {
                        if constexpr (Cfg::PACKED || Cfg::IDX) S.el[0][i] |= (typename Cfg::E)(j << w.sbits);
                        else S.key[0][i] |= j << w.sbits;
                    }
                }
            }
            __syncthreads();
            int cur;
            if constexpr (Cfg::PACKED || Cfg::IDX) cur = Sort::sort(S, (int)n, (int)(w.sbits + gbits), (int)w.sort_mode, w.status);
            else cur = Sort::sort(S, (int)n, (int)(w.sbits + gbits));
            auto Kc = [&S, cur](int i) -> uint32_t {
                if constexpr (Cfg::PACKED || Cfg::IDX) return Sort::key_of(S.el[cur][i]);
                else return S.key[cur][i];
            };
            const uint64_t* vsrc = src_v64 + start;
            auto Vc = [&S, cur, vsrc](int i) -> unsigned long long {
                if constexpr (Cfg::PACKED) {
                    return (unsigned long long)Sort::val_of(S.el[cur][i]);
                } else if constexpr (Cfg::IDX) {
                    return (unsigned long long)vsrc[(uint32_t)(S.el[cur][i] >> 32)];
                } else {
                    if constexpr (HAS_CNT) return (unsigned long long)S.val[cur][i];
                    else return 1ull;
                }
            };
            const int wch = ((((int)n + W - 1) / W) + 31) & ~31;
            const int w0 = min((int)n, warp * wch), w1 = min((int)n, w0 + wch);
            // 32-bit sums suffice when no run can reach 2^32
            const bool wide = __syncthreads_or(vmax > (0xFFFFFFFFull / (unsigned long long)n));
            uint32_t* ok_ = w.tmp_key + start;
            unsigned long long* ov = (unsigned long long*)(w.tmp_val + start);
            auto put_tmp = [&](bool wr, uint32_t pos, uint32_t k, unsigned long long v) {
                // site 109: a key of the leaf's runs
                if (wr && in_bounds(w.status, pos, n, 109)) { ok_[pos] = k; ov[pos] = v; }
            };

            uint32_t n_out;
            if (fuse) {
                if (!wide)
                    n_out = leaf_runs<uint32_t, W>(Kc, Vc, (int)n, w0, w1, s_any_zero != 0, pre, put_fused, s_run0,
                                                   s_nz, reinterpret_cast<uint32_t*>(s_carry), &s_tot);
                else
                    n_out = leaf_runs<unsigned long long, W>(Kc, Vc, (int)n, w0, w1, s_any_zero != 0, pre, put_fused,
                                                             s_run0, s_nz, s_carry, &s_tot);
                post(n_out);
            } else {
                auto no_pre = [](uint32_t) {};
                if (!wide)
                    n_out = leaf_runs<uint32_t, W>(Kc, Vc, (int)n, w0, w1, s_any_zero != 0, no_pre, put_tmp, s_run0,
                                                   s_nz, reinterpret_cast<uint32_t*>(s_carry), &s_tot);
                else
                    n_out = leaf_runs<unsigned long long, W>(Kc, Vc, (int)n, w0, w1, s_any_zero != 0, no_pre, put_tmp,
                                                             s_run0, s_nz, s_carry, &s_tot);
            }
            if (threadIdx.x == 0) w.leaf_d[l] = n_out;
            __syncthreads();
        } else if constexpr (Cfg::DENSE) {
            // oversized sub-bin (one group): dense shared-memory windows over
            // the subkey range, each compacted in key order
            unsigned long long* dense = reinterpret_cast<unsigned long long*>(smem_raw);
            uint32_t mn = 0xFFFFFFFFu, mx = 0;
            for (uint32_t i = start + threadIdx.x; i < end; i += THREADS) {
                uint32_t k;
                unsigned long long v;
                rec(i, k, v);
                mn = min(mn, k); mx = max(mx, k);
            }
            for (int o = 16; o > 0; o >>= 1) {
                mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
                mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            }
            if (threadIdx.x == 0) { red[0] = 0xFFFFFFFFull; red[1] = 0; }
            __syncthreads();
            if (lane == 0) {
                atomicMin(&red[0], (unsigned long long)mn);
                atomicMax(&red[1], (unsigned long long)mx);
            }
            __syncthreads();
            const uint32_t kmin = (uint32_t)red[0], kmax = (uint32_t)red[1];
            __syncthreads();
            uint32_t out = 0;
            constexpr int WD = Cfg::WD;
            constexpr int DEPT = WD / THREADS;
            for (uint64_t wlo = kmin; wlo <= kmax; wlo += WD) {
                for (int j = threadIdx.x; j < WD; j += THREADS) dense[j] = 0;
                __syncthreads();
                for (uint32_t i = start + threadIdx.x; i < end; i += THREADS) {
                    uint32_t k;
                    unsigned long long v;
                    rec(i, k, v);
                    if (k >= wlo && (uint64_t)k < wlo + WD) atomicAdd(&dense[k - wlo], v);
                }
                __syncthreads();
                uint32_t nz = 0;
                for (int j = 0; j < DEPT; ++j) nz += dense[j * THREADS + threadIdx.x] != 0;
                // order: the window is compacted in key order, row by row
                uint32_t tot = 0;
                for (int j = 0; j < DEPT; ++j) {
                    const int q = j * THREADS + threadIdx.x;
                    const unsigned long long v = dense[q];
                    uint32_t rt;
                    const uint32_t pos = block_exclusive_scan<uint32_t, THREADS>(v != 0, sw, &rt);
                    if (v) {
                        w.tmp_key[start + out + tot + pos] = (uint32_t)(wlo + q);
                        w.tmp_val[start + out + tot + pos] = v;
                    }
                    tot += rt;
                }
                (void)nz;
                out += tot;
                __syncthreads();
            }
            if (fuse) copy_fused(out);
            if (threadIdx.x == 0) w.leaf_d[l] = out;
            __syncthreads();
        }
    }
    if constexpr (Cfg::CAN_FUSE) {
        if (fuse) flush();
    }
}

template <int THREADS, int CAP, bool HAS_CNT, typename V, bool HASH>
static void launch_leaf(const AggWork& w, cudaStream_t s, int sms, int per_sm, uint32_t n_lo = 0,
                        uint32_t n_hi = 0xFFFFFFFFu) {
    using Cfg = LeafCfg<THREADS, CAP, HAS_CNT, V, HASH>;
    set_smem_limit((const void*)k_leaf<THREADS, CAP, HAS_CNT, V, HASH>, (int)Cfg::SMEM);
    k_leaf<THREADS, CAP, HAS_CNT, V, HASH><<<sms * per_sm, THREADS, Cfg::SMEM, s>>>(w, n_lo, n_hi);
}


// With small_leaves, leaves of at most SMALL_LEAF_CAP records go to a kernel
// of small CTAs (many CTAs per SM hide the fixed cost per leaf, which
// dominates when contexts hold a few samples each), the others to the leaf
// capacity's kernel.
template <bool HASH>
static void launch_packed_leaves(const AggWork& w, cudaStream_t s, int sms) {
    const uint32_t lo = w.small_leaves ? SMALL_LEAF_CAP + 1 : 0;
    if (w.has_cnt) {
        if (w.small_leaves) launch_leaf<SMALL_LEAF_THREADS, SMALL_LEAF_CAP, true, uint32_t, HASH>(w, s, sms, 8, 0, SMALL_LEAF_CAP);
        if (w.cap == LEAF_CAP_LARGE) launch_leaf<LEAF_THREADS_LARGE, LEAF_CAP_LARGE, true, uint32_t, HASH>(w, s, sms, 1, lo);
        else launch_leaf<256, LEAF_CAP_SMALL, true, uint32_t, HASH>(w, s, sms, 2, lo);
    } else {
        if (w.small_leaves) launch_leaf<SMALL_LEAF_THREADS, SMALL_LEAF_CAP, false, uint32_t, HASH>(w, s, sms, 8, 0, SMALL_LEAF_CAP);
        if (w.cap == LEAF_CAP_LARGE) launch_leaf<LEAF_THREADS_LARGE, LEAF_CAP_LARGE, false, uint32_t, HASH>(w, s, sms, 1, lo);
        else launch_leaf<256, LEAF_CAP_SMALL, false, uint32_t, HASH>(w, s, sms, 2, lo);
    }
}

void launch_leaves(const AggWork& w, cudaStream_t s, int sms, uint64_t* launches) {
    if (w.val64) {
        launch_leaf<256, LEAF_CAP_SMALL, true, uint64_t, false>(w, s, sms, 2);
        *launches += 1;
        return;
    }
    if (w.leaf_hash) launch_packed_leaves<true>(w, s, sms);
    else launch_packed_leaves<false>(w, s, sms);
    *launches += 1 + (w.small_leaves ? 1 : 0);
}

}  // namespace hpa
