// Internal declarations shared by the host orchestration (hpa_host.cu) and
// the kernel translation units.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "hpa_dev.cuh"

namespace hpa {

// One sample buffer of an aggregation call, as the kernels read it.
struct BufDev {
    const uint64_t* pc;
    const uint32_t* ctx;
    const uint8_t* stall;
    const uint32_t* count;      // may be null (every record counts 1)
    uint64_t n;
    uint64_t tile_base;         // first global tile of this buffer
    uint32_t n_ctx;
    uint32_t n_stall;
    uint32_t grp_base;          // first global group (group = grp_base + ctx)
    uint32_t bin;               // index into the DevBinary table
    uint32_t first_leaf_item;   // (filled on device) unused by the host
    uint32_t pad;
    uint64_t part_base;         // first global part of this buffer (partition path)
    uint64_t cnt_base;          // first part counter of this buffer: sum of bins * parts before it
    uint32_t seg_base;          // first bucket segment of this buffer (part_mode 2)
    uint32_t pad2;
    uint64_t* total;            // per-stall totals (may be null)
    uint64_t* unknown;
    // outputs
    uint32_t* key_ctx;
    uint32_t* key_node;
    uint8_t* key_stall;
    uint64_t* val;
    uint64_t* n_keys;
    uint64_t capacity;
};

// Scratch of one aggregation call (device pointers).
struct AggWork {
    uint32_t G;            // groups (sum of n_ctx)
    uint32_t n_buf;
    uint64_t n_tiles;
    uint32_t cap;          // leaf capacity
    uint32_t q;            // cap / 2
    uint32_t sb;           // stall bits
    uint32_t sbits;        // subkey bits (node bits + stall bits)
    uint32_t span_log;     // at most 2^span_log groups per item (32 - sbits)
    uint32_t L_max;        // leaf table capacity
    uint32_t has_cnt;
    uint32_t* grp_hist;    // [G+1] -> exclusive scan -> seg_off
    uint32_t* grp_cursor;  // [G << cur_shift] scatter cursors, one per 2^cur_shift words
    uint32_t cur_shift;
    uint32_t sort_mode;    // leaf radix ranking: 0 by digit width, 1 match_any, 2 ballots, 3 alternate
    uint32_t* item_id;     // [G+1] flags -> exclusive scan
    uint32_t* item_grp0;   // [G]
    uint32_t* item_nleaf;  // [G+1] -> exclusive scan -> leaf_base
    uint32_t* leaf_start;  // [L_max]
    uint32_t* leaf_end;    // [L_max]
    uint32_t* leaf_grp0;   // [L_max]
    uint32_t* leaf_info;   // [L_max] bit0: records in rec2; bits 8..: buffer index
    uint32_t* leaf_d;      // [L_max+1] -> exclusive scan -> leaf_out
    uint32_t* buf_first_leaf;     // [n_buf + 1]
    unsigned long long* buf_bad;  // [n_buf]
    uint32_t val64;        // record values are uint64 (rec_v64) instead of uint32 (rec_cnt)
    uint32_t* rec_sub;     // [N]
    uint32_t* rec_cnt;     // [N] (if has_cnt and !val64)
    uint32_t* rec2_sub;    // [N]
    uint32_t* rec2_cnt;    // [N]
    uint64_t* rec_v64;     // [N] (if val64)
    uint64_t* rec2_v64;    // [N]
    uint2* rec_pair;       // [N] {subkey, count} (if has_cnt and !val64; rec_sub unused then)
    uint2* rec2_pair;      // [N]
    uint32_t* tmp_key;     // [N]
    uint64_t* tmp_val;     // [N]
    uint64_t n_rec;        // N: entries of each record array above
    uint32_t* scan_tmp;    // device-wide scan partials
    const BufDev* bufs;    // [n_buf]
    const uint64_t* buf_tile;     // [n_buf + 1] tile prefix
    const uint32_t* buf_grp;      // [n_buf + 1] group prefix
    const DevBinary* bins;
    DevStatus* status;
    // partition path (every buffer's contexts fit in shared memory)
    uint32_t part_mode;           // 0 per-context cursors, 1 bins = contexts, 2 bins = buckets + second pass
    uint32_t part_ctx_max;        // largest number of bins of a buffer
    uint32_t part_shift;          // a bin holds 2^part_shift consecutive contexts
    uint32_t n_seg;               // part_mode 2: bucket segments of the call
    const uint32_t* buf_seg;      // [n_buf + 1] segment prefix
    uint32_t* seg_chunk;          // [n_seg + 1] chunks per segment -> exclusive scan
    uint32_t* cnt2;               // [n_cnt2 + 1] second-pass counters -> exclusive scan
    uint64_t n_cnt2;              // upper bound of the second-pass counters
    uint8_t* rec2_dig;            // [N] low context bits of the bucket-grouped records
    uint64_t part_len;            // samples per part
    uint64_t n_parts;
    uint64_t n_cnt;               // part counters: sum over buffers of n_ctx * parts
    const uint64_t* buf_part;     // [n_buf + 1] part prefix
    uint32_t* part_cnt;           // [n_cnt + 1] counts -> exclusive scan -> first record positions
    uint32_t emit_totals;         // k_emit sums the per-stall and UNKNOWN totals
    uint32_t small_leaves;        // leaves of <= SMALL_LEAF_CAP records go to the small-leaf kernel
    uint32_t leaf_hash;           // leaves aggregate in a shared-memory hash table before sorting
    uint32_t timeout_iters;       // polls of a bounded device wait (0 = 1 << 22)
    // fused leaves: each leaf writes its keys to the output arrays itself, at
    // an offset found by a look-back over the leaves before it (k_emit is
    // then not launched); leaves are taken in index order from leaf_ticket
    uint32_t fuse_emit;
    uint32_t emit_separate;          // 1: never fused (every leaf goes through k_emit)
    unsigned long long* leaf_look;   // [L_max] look-back words (zeroed per call)
    uint32_t* leaf_ticket;           // [1] next leaf to take (zeroed per call)
};

// look-back words of fused leaves: a count (AGG) or an inclusive prefix
// (INCL) in the low bits; DIRECT marks a leaf that wrote its keys itself
constexpr unsigned long long LOOK_AGG = 1ull << 62, LOOK_INCL = 1ull << 63, LOOK_DIRECT = 1ull << 61,
                             LOOK_VAL = (1ull << 61) - 1;
constexpr uint32_t LOOK_QUICK = 2;       // polls a fused leaf makes before it leaves its keys to k_emit

constexpr int TILE = 4096;            // samples per tile of the sample-reading kernels
constexpr uint32_t HPA_MAX_STALL_DEV = 32;
constexpr uint32_t HIST_SMEM_MAX = 24576;    // contexts counted in shared memory (96 KB)
constexpr uint32_t LEAF_CAP_SMALL = 4096;   // 256 threads, two CTAs per SM
constexpr uint32_t LEAF_CAP_LARGE = 10240;  // 512 threads, one CTA per SM
constexpr int LEAF_THREADS_LARGE = 512;
constexpr uint32_t SMALL_LEAF_CAP = 1024;    // leaves up to this size run in 128-thread CTAs, 8 per SM
constexpr int SMALL_LEAF_THREADS = 128;
constexpr uint32_t BIG_FINE_MAX_LOG = 14;   // at most 2^14 fine bins per big group (64 KB counters)
constexpr int BIG_THREADS = 512;
constexpr int BIG_EPT = ((1 << BIG_FINE_MAX_LOG) + 1 + BIG_THREADS - 1) / BIG_THREADS;
constexpr int PART_THREADS = 512;
constexpr int PART_U = 8;                    // records in flight per thread in k_part2_scatter (4: +0.13 ms on the large profile)
constexpr int PART_TILE = PART_THREADS * PART_U;   // records staged per tile in k_part2_scatter
// k_part_scatter (attribution + first partition pass): CTA size, samples in
// flight per thread, CTAs per SM
constexpr int PSC_THREADS = 512;
constexpr int PSC_U = 4;
constexpr int PSC_MIN_BLOCKS = 2;
constexpr int PSC_TILE = PSC_THREADS * PSC_U;
constexpr uint32_t PART_CTX_MAX = 4096;      // contexts per buffer on the partition path; with more, the
                                             // (context, part) regions written at once overflow L2 and the
                                             // per-context cursor path is faster
constexpr uint64_t PART_CNT_MAX = 1ull << 26; // part counters per call on the partition path
constexpr int PART_SCAN_EPT = (int)((PART_CTX_MAX + 1 + PART_THREADS - 1) / PART_THREADS);
constexpr int PSC_SCAN_EPT = (int)((PART_CTX_MAX + 1 + PSC_THREADS - 1) / PSC_THREADS);
constexpr uint32_t PART2_CTX_MAX = 65536;    // contexts per buffer on the two-level partition path
constexpr uint64_t PART2_LEN = 32768;        // records per chunk of the second pass
constexpr int SCAN_THREADS = 512;
constexpr int SCAN_EPT = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_EPT;

// Raise the dynamic shared-memory limit of kernel `fn` to at least `bytes`
// on the current device.  The attribute belongs to one device; the largest
// limit set per (kernel, device) is remembered under a lock (calls may come
// from several host threads and handles on several devices), and a limit is
// never lowered, so launches of any smaller size stay valid.
void set_smem_limit(const void* fn, int bytes);

// device-wide exclusive scan of n uint32 values (in place allowed);
// out[n] receives the total.  tmp needs scan_tmp_words(n) words.
size_t scan_tmp_words(uint64_t n);
void scan_u32(const uint32_t* in, uint32_t* out, uint64_t n, uint32_t* tmp, cudaStream_t s, uint64_t* launches);

// aggregation pipeline (A1 + A2) over a prepared AggWork
constexpr int N_PHASES = 5;
// ev (may be null): N_PHASES + 1 events recorded at the phase boundaries
void run_aggregate(const AggWork& w, cudaStream_t s, int sms, uint64_t* launches, cudaEvent_t* ev);

// Keys of a profile expanded to every structure ancestor (inclusive metrics
// over the structure tree): each key (ctx, node, stall, val) yields one record
// per node on the path node -> function node; UNKNOWN yields itself only.
struct ExpandSrc {
    const uint32_t* ctx;
    const uint32_t* node;
    const uint8_t* stall;
    const uint64_t* val;
    const uint64_t* n_keys;   // device count of keys
    uint64_t cap;             // host bound on the key count
    const uint32_t* parent;   // structure tree
    const uint32_t* depth;    // depth of each node (FUNC = 0)
    uint32_t M;               // n_nodes (UNKNOWN is coded as M)
    uint32_t n_ctx;
};
void run_expand_aggregate(const AggWork& w, const ExpandSrc& x, cudaStream_t s, int sms, uint64_t* launches);

// the aggregation's tail after the records are grouped: big-group split,
// leaves, key placement and the per-buffer key counts
void run_group_tail(const AggWork& w, cudaStream_t s, int sms, uint64_t* launches);

// zero every buffer's per-stall totals (device-side, so a captured graph
// reads the current descriptors)

// shared stages for other producers
void clear_work(const AggWork& w, cudaStream_t s, bool totals = false);   // totals: the buffers' too
void run_plan(const AggWork& w, cudaStream_t s, int sms, uint64_t* launches, bool seg_ready, bool part_seg = false);
void launch_big_partition(const AggWork& w, cudaStream_t s, int sms, uint64_t* launches);
// every leaf kernel of one aggregation (hpa_leaf.cu)
void launch_leaves(const AggWork& w, cudaStream_t s, int sms, uint64_t* launches);
void launch_finalize(const AggWork& w, cudaStream_t s, uint64_t* launches);

// largest b with pre[b] <= x (pre non-decreasing, pre[0] = 0)
template <typename T>
__device__ __forceinline__ uint32_t upper_index(const T* pre, uint32_t n, T x) {
    uint32_t lo = 0, hi = n;
    while (hi - lo > 1) {
        const uint32_t m = (lo + hi) >> 1;
        if (pre[m] <= x) lo = m; else hi = m;
    }
    return lo;
}

}  // namespace hpa
