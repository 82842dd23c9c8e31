// Attribution (Sections 4.2, 5) and raw-metric aggregation (Section 4.5) of
// GPU PC samples on sm_103a.
//
// Pipeline over one or many sample buffers (a "group" is one launch context
// of one buffer; records of a group are aggregated together):
//   k_grp_hist       records per group (reads ctx only)
//   scan             group offsets
//   k_item_flags,    groups are packed into items of <= cap records (runs of
//   k_items, ...     small groups, or one group); a group with more than cap
//                    records becomes a "big" item split into 2^h sub-bins
//   k_attribute      reads every sample once, attributes its PC to a
//                    structure node, packs (node, stall) into a subkey and
//                    stores (subkey, count) in sample order
//   k_scatter        moves each record into its group's segment
//   k_big_partition  splits big groups into fine bins (top subkey bits) and
//                    cuts the bins into leaves of at most cap records
//   k_leaf           per leaf (hpa_leaf.cu): shared-memory radix sort + run
//                    reduction, hash aggregation, or dense windows for
//                    oversized sub-bins
//   scan + k_emit    leaves are in key order; their run counts give every
//                    key's output position
//   k_finalize       per-buffer key counts and status
// Counts are summed exactly in 64-bit integers; keys come out ascending by
// (ctx, node, stall).

#include <algorithm>
#include <map>
#include <mutex>
#include <type_traits>

#include "hpa_bulk.cuh"
#include "hpa_internal.h"

namespace hpa {

// ------------------------------------------------------------------ scans
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_reduce(const uint32_t* in, uint64_t n, uint32_t* part) {
    __shared__ uint32_t sw[33];
    const uint64_t base = (uint64_t)blockIdx.x * SCAN_TILE + (uint64_t)threadIdx.x * SCAN_EPT;
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_EPT; ++i)
        if (base + i < n) s += in[base + i];
    s = warp_sum(s);
    if (lane_id() == 0) sw[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        uint32_t v = threadIdx.x < SCAN_THREADS / 32 ? sw[threadIdx.x] : 0;
        v = warp_sum(v);
        if (threadIdx.x == 0) part[blockIdx.x] = v;
    }
}

__global__ void __launch_bounds__(1024) k_scan_partials(uint32_t* part, uint32_t nb) {
    __shared__ uint32_t sw[33];
    uint32_t carry = 0;
    for (uint32_t base = 0; base < nb; base += 1024) {
        const uint32_t i = base + threadIdx.x;
        const uint32_t v = i < nb ? part[i] : 0;
        uint32_t tot;
        const uint32_t e = block_exclusive_scan<uint32_t, 1024>(v, sw, &tot);
        if (i < nb) part[i] = carry + e;
        carry += tot;
    }
    if (threadIdx.x == 0) part[nb] = carry;
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_down(const uint32_t* in, uint32_t* out, uint64_t n,
                                                            const uint32_t* part, uint32_t nb) {
    __shared__ uint32_t sw[33];
    const uint64_t base = (uint64_t)blockIdx.x * SCAN_TILE + (uint64_t)threadIdx.x * SCAN_EPT;
    uint32_t v[SCAN_EPT];
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_EPT; ++i) {
        v[i] = (base + i < n) ? in[base + i] : 0;
        s += v[i];
    }
    uint32_t tot;
    uint32_t pre = block_exclusive_scan<uint32_t, SCAN_THREADS>(s, sw, &tot) + part[blockIdx.x];
#pragma unroll
    for (int i = 0; i < SCAN_EPT; ++i) {
        if (base + i < n) out[base + i] = pre;
        pre += v[i];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = part[nb];
}

void set_smem_limit(const void* fn, int bytes) {
    static std::mutex mu;
    static std::map<std::pair<const void*, int>, int> limit;   // largest limit set per (kernel, device)
    if (bytes <= 48 * 1024) return;                             // within the default limit
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(mu);
    int& cur = limit[std::make_pair(fn, dev)];
    if (bytes <= cur) return;                                   // the limit only ever grows
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) == cudaSuccess) cur = bytes;
    else cudaGetLastError();
}

// Arrays of up to SCAN_ONE_CTA_MAX entries: one CTA scans them in one launch
// (where the three-kernel scan pays three launch gaps).  A single CTA is
// latency-bound beyond that: 1.4-2.4 x 10^5 entries took 0.13-0.6 ms in one
// CTA, 16,384 at a time, against a few microseconds for the three kernels.
constexpr int SCAN_SMALL_THREADS = 1024, SCAN_SMALL_EPT = 16;
constexpr uint64_t SCAN_ONE_CTA_MAX = (uint64_t)SCAN_SMALL_THREADS * SCAN_SMALL_EPT;

// exclusive scan of in[0, n), n <= SCAN_ONE_CTA_MAX, into out[0, n) by one
// CTA of SCAN_SMALL_THREADS threads, the total in out[n] (in == out allowed)
__device__ void cta_scan_u32(const uint32_t* in, uint32_t* out, uint32_t n, uint32_t* sw) {
    const uint32_t base = threadIdx.x * SCAN_SMALL_EPT;
    uint32_t v[SCAN_SMALL_EPT];
    uint32_t sum = 0;
#pragma unroll
    for (int i = 0; i < SCAN_SMALL_EPT; ++i) {
        v[i] = base + i < n ? in[base + i] : 0u;
        sum += v[i];
    }
    uint32_t tot;
    uint32_t pre = block_exclusive_scan<uint32_t, SCAN_SMALL_THREADS>(sum, sw, &tot);
#pragma unroll
    for (int i = 0; i < SCAN_SMALL_EPT; ++i) {
        if (base + i < n) out[base + i] = pre;
        pre += v[i];
    }
    if (threadIdx.x == 0) out[n] = tot;
}

__global__ void __launch_bounds__(SCAN_SMALL_THREADS) k_scan_small(const uint32_t* in, uint32_t* out, uint32_t n) {
    __shared__ uint32_t sw[33];
    cta_scan_u32(in, out, n, sw);
}

size_t scan_tmp_words(uint64_t n) { return (size_t)((n + SCAN_TILE - 1) / SCAN_TILE) + 2; }

void scan_u32(const uint32_t* in, uint32_t* out, uint64_t n, uint32_t* tmp, cudaStream_t s, uint64_t* launches) {
    if (n <= SCAN_ONE_CTA_MAX) {
        k_scan_small<<<1, SCAN_SMALL_THREADS, 0, s>>>(in, out, (uint32_t)n);
        *launches += 1;
        return;
    }
    const uint32_t nb = (uint32_t)std::max<uint64_t>(1, (n + SCAN_TILE - 1) / SCAN_TILE);
    k_scan_reduce<<<nb, SCAN_THREADS, 0, s>>>(in, n, tmp);
    k_scan_partials<<<1, 1024, 0, s>>>(tmp, nb);
    k_scan_down<<<nb, SCAN_THREADS, 0, s>>>(in, out, n, tmp, nb);
    *launches += 3;
}

// ------------------------------------------------------------------ helpers
// A big group (more than cap records) is split by fine bins: the top h bits
// of its subkey.  A bin spans 2^(sbits - h) subkeys; h is chosen so that this
// is at most one dense window of the leaf (2^13 subkeys) whenever 2^14 bins
// allow it, so a bin that alone exceeds cap is reduced in one dense pass.
__device__ __forceinline__ uint32_t fine_bits(uint32_t sbits) {
    const uint32_t h = sbits > 13 ? sbits - 13 : 0;
    return min(sbits, min((uint32_t)BIG_FINE_MAX_LOG, max(12u, h)));
}

// Leaves of a big group of n records are runs of consecutive fine bins: a
// leaf starts at the first bin, at every bin whose offset enters a new window
// of q records, and at every bin of more than q records.  That is at most
// 1 + floor(n / q) + floor(n / (q + 1)) <= 2 ceil(n / q) starts, and a leaf of
// bins of at most q records each holds fewer than 2q = cap records.
__device__ __forceinline__ uint32_t big_leaf_slots(uint32_t n, uint32_t q) { return 2 * ((n + q - 1) / q); }

__device__ __forceinline__ bool big_leaf_head(const uint32_t* off, uint32_t j, uint32_t q) {
    return j == 0 || off[j] / q != off[j - 1] / q || off[j + 1] - off[j] > q;
}

// ------------------------------------------------------------------ K1: records per group
// Each CTA takes a contiguous run of tiles.  A buffer with at most
// HIST_SMEM_MAX contexts is counted in shared memory and flushed when the
// CTA leaves that buffer; larger context spaces count in global memory.
__global__ void __launch_bounds__(256) k_grp_hist(AggWork w) {
    extern __shared__ uint32_t sh[];
    const uint64_t per = (w.n_tiles + gridDim.x - 1) / gridDim.x;
    const uint64_t t0 = blockIdx.x * per, t1 = min(w.n_tiles, t0 + per);
    uint32_t cur_b = 0xFFFFFFFFu, cur_n = 0, cur_base = 0;
    bool priv = false;
    auto flush = [&]() {
        if (priv) {
            __syncthreads();
            for (uint32_t c = threadIdx.x; c < cur_n; c += blockDim.x)
                if (sh[c]) atomicAdd(&w.grp_hist[cur_base + c], sh[c]);
            __syncthreads();
        }
    };
    for (uint64_t t = t0; t < t1; ++t) {
        const uint32_t b = upper_index<uint64_t>(w.buf_tile, w.n_buf, t);
        const BufDev& B = w.bufs[b];
        if (b != cur_b) {
            flush();
            cur_b = b; cur_n = B.n_ctx; cur_base = B.grp_base;
            priv = cur_n <= HIST_SMEM_MAX;
            if (priv) {
                for (uint32_t c = threadIdx.x; c < cur_n; c += blockDim.x) sh[c] = 0;
                __syncthreads();
            }
        }
        const uint64_t i0 = (t - B.tile_base) * TILE;
        const uint64_t i1 = min(i0 + TILE, B.n);
        const uint32_t* ctx = B.ctx;
        uint32_t bad = 0;
        auto count = [&](uint32_t c) {
            if (c >= cur_n) { ++bad; return; }
            if (priv) atomicAdd(&sh[c], 1u);
            else atomicAdd(&w.grp_hist[cur_base + c], 1u);
        };
        if (i1 - i0 == TILE && (((uintptr_t)(ctx + i0)) & 15) == 0) {
            // full aligned tile: 16 contexts per thread in four 16-byte loads
            const uint4* v = reinterpret_cast<const uint4*>(ctx + i0);
            uint4 q[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) q[k] = ld_stream(&v[k * 256 + threadIdx.x]);
#pragma unroll
            for (int k = 0; k < 4; ++k) { count(q[k].x); count(q[k].y); count(q[k].z); count(q[k].w); }
        } else {
            for (uint64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) count(ld_stream(&ctx[i]));
        }
        if (bad) atomicAdd(&w.buf_bad[b], (unsigned long long)bad);
    }
    flush();
}

// ------------------------------------------------------------------ K3..K8: items and leaves
// Each step is a loop over groups or items from `i0` in steps of `step`:
// one thread per element across a grid (the kernels below), or the threads
// of one CTA (k_plan_one, for calls with few groups).
__device__ __forceinline__ void item_flags_range(const AggWork& w, uint32_t i0, uint32_t step) {
    const uint32_t* seg = w.grp_hist;
    const uint32_t span_mask = (w.span_log >= 32) ? 0xFFFFFFFFu : ((1u << w.span_log) - 1);
    for (uint32_t g = i0; g < w.G; g += step) {
        const uint32_t s0 = seg[g];
        uint32_t f = 0;
        if (g == 0) {
            f = 1;
        } else {
            const uint32_t sp = seg[g - 1];
            const uint32_t ng = seg[g + 1] - s0, np = s0 - sp;
            if (ng > w.q || np > w.q) f = 1;
            if (s0 / w.q != sp / w.q) f = 1;
            if ((g & span_mask) == 0) f = 1;
            if (w.n_buf > 1) {
                const uint32_t b = upper_index<uint32_t>(w.buf_grp, w.n_buf, g);
                if (w.buf_grp[b] == g) f = 1;
            }
        }
        w.item_id[g] = f;
        w.grp_cursor[(size_t)g << w.cur_shift] = s0;
    }
}

__device__ __forceinline__ void items_range(const AggWork& w, uint32_t i0, uint32_t step) {
    for (uint32_t g = i0; g < w.G; g += step)
        if (w.item_id[g + 1] != w.item_id[g]) w.item_grp0[w.item_id[g]] = g;
}

__device__ __forceinline__ void items_size_range(const AggWork& w, uint32_t i0, uint32_t step) {
    const uint32_t n_items = w.item_id[w.G];
    const uint32_t* seg = w.grp_hist;
    for (uint32_t it = i0; it < w.G; it += step) {
        uint32_t nl = 0;
        if (it < n_items) {
            const uint32_t g0 = w.item_grp0[it];
            const uint32_t g1 = (it + 1 < n_items) ? w.item_grp0[it + 1] : w.G;
            const uint32_t n = seg[g1] - seg[g0];
            nl = (n > w.cap) ? big_leaf_slots(n, w.q) : 1u;
        }
        w.item_nleaf[it] = nl;
    }
}

__device__ __forceinline__ void leaves_range(const AggWork& w, uint32_t i0, uint32_t step) {
    const uint32_t n_items = w.item_id[w.G];
    const uint32_t* seg = w.grp_hist;
    const uint32_t* leaf_base = w.item_nleaf;
    for (uint32_t it = i0; it < n_items; it += step) {
        const uint32_t g0 = w.item_grp0[it];
        const uint32_t g1 = (it + 1 < n_items) ? w.item_grp0[it + 1] : w.G;
        const uint32_t n = seg[g1] - seg[g0];
        const uint32_t l = leaf_base[it];
        const uint32_t b = upper_index<uint32_t>(w.buf_grp, w.n_buf, g0);
        if (w.buf_grp[b] == g0) w.buf_first_leaf[b] = l;
        if (n <= w.cap) {
            w.leaf_start[l] = seg[g0];
            w.leaf_end[l] = seg[g1];
            w.leaf_grp0[l] = g0;
            w.leaf_info[l] = b << 8;
        }
    }
    if (i0 == 0) w.buf_first_leaf[w.n_buf] = leaf_base[w.G];
}

// group offsets (exclusive) from the scanned part counts (partition path, part_mode 1)
__device__ __forceinline__ void part_seg_range(const AggWork& w, uint32_t i0, uint32_t step) {
    for (uint32_t g = i0; g <= w.G; g += step) {
        if (g == w.G) { w.grp_hist[g] = w.part_cnt[w.n_cnt]; continue; }
        const uint32_t b = upper_index<uint32_t>(w.buf_grp, w.n_buf, g);
        const BufDev& B = w.bufs[b];
        const uint64_t parts = w.buf_part[b + 1] - w.buf_part[b];
        w.grp_hist[g] = w.part_cnt[B.cnt_base + (uint64_t)(g - B.grp_base) * parts];
    }
}

#define HPA_GRID_RANGE blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x
__global__ void k_item_flags(AggWork w) { item_flags_range(w, HPA_GRID_RANGE); }
__global__ void k_items(AggWork w) { items_range(w, HPA_GRID_RANGE); }
__global__ void k_items_size(AggWork w) { items_size_range(w, HPA_GRID_RANGE); }
__global__ void k_leaves(AggWork w) { leaves_range(w, HPA_GRID_RANGE); }
__global__ void k_part_seg(AggWork w) { part_seg_range(w, HPA_GRID_RANGE); }
#undef HPA_GRID_RANGE

// The whole plan in one CTA (calls with fewer than SCAN_ONE_CTA_MAX groups,
// so that each of its scans is one CTA's): group offsets (from the part
// counts, or a scan of the group histogram), item flags, their scan, items,
// leaf slots per item, their scan, leaves -- one launch for seven.
constexpr uint32_t PLAN_ONE_CTA_MAX = (uint32_t)SCAN_ONE_CTA_MAX - 1;

__global__ void __launch_bounds__(SCAN_SMALL_THREADS) k_plan_one(AggWork w, int seg_mode) {
    __shared__ uint32_t sw[33];
    const uint32_t t = threadIdx.x, n = blockDim.x;
    if (seg_mode == 1) part_seg_range(w, t, n);
    else if (seg_mode == 0) cta_scan_u32(w.grp_hist, w.grp_hist, w.G, sw);
    __syncthreads();
    item_flags_range(w, t, n);
    __syncthreads();
    cta_scan_u32(w.item_id, w.item_id, w.G, sw);
    __syncthreads();
    items_range(w, t, n);
    __syncthreads();
    items_size_range(w, t, n);
    __syncthreads();
    cta_scan_u32(w.item_nleaf, w.item_nleaf, w.G, sw);
    __syncthreads();
    leaves_range(w, t, n);
}

// ------------------------------------------------------------------ K9a: attribute
// U samples per thread: the structure node of each PC (Section 4.2) through
// the direct-answer directory, with a short forward walk over the table
// entries where a directory bucket straddles several of them (the entry
// holding the bucket start and the next one are loaded together; the last
// entry, at the span, ends every walk).  Only these loads are dependent, so
// U lookups per thread stay in flight.
template <int U>
__device__ __forceinline__ void lookup_nodes(const DevBinary& bin, const uint64_t (&pc)[U], const bool (&ok)[U],
                                             uint32_t (&nd)[U], uint64_t keep, DevStatus* st) {
    uint32_t off[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        nd[u] = bin.n_nodes;
        off[u] = 0;
        if (ok[u]) {
            const uint64_t o = pc[u] - bin.pc_base;
            if (o < bin.span) {
                off[u] = (uint32_t)o;
                // site 111: directory entry
                if (in_bounds(st, off[u] >> bin.dshift, bin.n_dir, 111))
                    nd[u] = ld_keep(&bin.dir[off[u] >> bin.dshift], keep);
            }
        }
    }
    // the first two entries of every walk are loaded for all U lookups
    // before any walk goes on, so that the U second-level loads overlap
    uint2 cur[U], nx[U];
    uint32_t j[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        if (nd[u] & DIR_SEARCH) {
            j[u] = nd[u] & ~DIR_SEARCH;
            if (!in_bounds(st, j[u] + 1, bin.n_ent, 112)) { nd[u] = bin.n_nodes; continue; }   // site 112: interval entry
            cur[u] = ld_keep2(&bin.ent[j[u]], keep);
            nx[u] = ld_keep2(&bin.ent[j[u] + 1], keep);
        }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
        if (nd[u] & DIR_SEARCH) {
            while (nx[u].x <= off[u]) {
                cur[u] = nx[u];
                ++j[u];
                if (!in_bounds(st, j[u] + 1, bin.n_ent, 112)) break;
                nx[u] = ld_keep2(&bin.ent[j[u] + 1], keep);
            }
            nd[u] = cur[u].y;
        }
    }
}

// Streams every sample once: attributes its PC, packs (node, stall) into a
// subkey and stores {subkey, count} in sample order (coalesced) in the
// second record buffer, for k_scatter.  Used when a buffer has more contexts
// than the partition path keeps in shared memory.
template <bool HAS_CNT, int U>
__global__ void __launch_bounds__(256, 4) k_attribute(AggWork w) {
    const uint32_t tid = threadIdx.x;
    const uint64_t keep = policy_evict_last();
    for (uint64_t t = blockIdx.x; t < w.n_tiles; t += gridDim.x) {
        const uint32_t b = upper_index<uint64_t>(w.buf_tile, w.n_buf, t);
        const BufDev B = w.bufs[b];
        const DevBinary bin = w.bins[B.bin];
        const uint64_t i0 = (t - B.tile_base) * TILE;
        const uint64_t i1 = min(i0 + TILE, B.n);
        const uint64_t stage0 = t * TILE - i0;               // staging index = stage0 + i
        uint32_t bad = 0;
        for (uint64_t base = i0 + tid; base < i1; base += 256 * U) {
            uint64_t pc[U];
            uint32_t st[U], cnt[U], nd[U];
            bool ok[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const uint64_t i = base + (uint64_t)u * 256;
                ok[u] = i < i1;
                pc[u] = 0; st[u] = 0; cnt[u] = 1u;
                if (ok[u]) {
                    st[u] = ld_stream(&B.stall[i]);
                    pc[u] = ld_stream((const unsigned long long*)&B.pc[i]);
                    if (HAS_CNT && B.count) cnt[u] = ld_stream(&B.count[i]);
                }
            }
            lookup_nodes<U>(bin, pc, ok, nd, keep, w.status);
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (!ok[u]) continue;
                const uint64_t i = base + (uint64_t)u * 256;
                const bool bad_stall = st[u] >= B.n_stall;
                const uint32_t sub = bad_stall ? 0u : ((nd[u] << w.sb) | st[u]);
                if (HAS_CNT) st_stream(&w.rec2_pair[stage0 + i], make_uint2(sub, bad_stall ? 0u : cnt[u]));
                else st_stream(&w.rec2_sub[stage0 + i], sub);
                bad += bad_stall;
            }
        }
        if (bad) atomicAdd(&w.buf_bad[b], (unsigned long long)bad);
    }
}

// ------------------------------------------------------------------ K9b: scatter by context
// Reads (ctx, staged record) in sample order and moves each record to its
// context's segment; the cursor atomic is the only dependent operation.
template <bool HAS_CNT, int U>
__global__ void __launch_bounds__(256) k_scatter(AggWork w) {
    for (uint64_t t = blockIdx.x; t < w.n_tiles; t += gridDim.x) {
        const uint32_t b = upper_index<uint64_t>(w.buf_tile, w.n_buf, t);
        const BufDev& B = w.bufs[b];
        const uint32_t n_ctx = B.n_ctx, gbase = B.grp_base;
        const uint32_t* ctx = B.ctx;
        const uint64_t i0 = (t - B.tile_base) * TILE;
        const uint64_t i1 = min(i0 + TILE, B.n);
        const uint64_t stage0 = t * TILE - i0;
        for (uint64_t base = i0 + threadIdx.x; base < i1; base += 256 * U) {
            uint32_t c[U];
            uint2 r[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const uint64_t i = base + (uint64_t)u * 256;
                c[u] = 0xFFFFFFFFu;
                if (i < i1) {
                    c[u] = ld_stream(&ctx[i]);
                    if (HAS_CNT) r[u] = ld_stream(&w.rec2_pair[stage0 + i]);
                    else r[u].x = ld_stream(&w.rec2_sub[stage0 + i]);
                }
            }
            uint32_t slot[U];
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (c[u] < n_ctx) slot[u] = atomicAdd(&w.grp_cursor[(size_t)(gbase + c[u]) << w.cur_shift], 1u);
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (c[u] >= n_ctx) continue;
                if (!in_bounds(w.status, slot[u], w.n_rec, 101)) continue;   // site 101: record slot
                if (HAS_CNT) w.rec_pair[slot[u]] = r[u];
                else w.rec_sub[slot[u]] = r[u].x;
            }
        }
    }
}

// ------------------------------------------------------------------ partition path
// For buffers whose contexts fit in shared memory, records are grouped by
// context without global atomics.  Each buffer is cut into parts of
// part_len samples; k_part_hist counts the valid records of every (bin,
// part) into part_cnt[cnt_base + bin * parts + part] (bin-major), one
// exclusive scan of part_cnt then gives the position of each (bin, part)'s
// first record in the bin-grouped record array, and k_part_scatter
// attributes every sample and places its record with a shared-memory cursor
// per bin.  With part_mode 1 a bin is a context and the group offsets are
// read off the scan.  With part_mode 2 (more contexts) a bin is a bucket of
// 2^part_shift consecutive contexts, the records land bucket-grouped in the
// second record buffer with their context's low bits in rec2_dig, and a
// second pass of the same shape groups each bucket by those bits.
__global__ void __launch_bounds__(PART_THREADS) k_part_hist(AggWork w) {
    extern __shared__ uint32_t sh[];
    for (uint64_t p = blockIdx.x; p < w.n_parts; p += gridDim.x) {
        const uint32_t b = upper_index<uint64_t>(w.buf_part, w.n_buf, p);
        const BufDev& B = w.bufs[b];
        const uint32_t n_ctx = B.n_ctx;
        const uint64_t pl = p - B.part_base;
        const uint64_t parts = w.buf_part[b + 1] - w.buf_part[b];
        const uint64_t i0 = pl * w.part_len, i1 = min(i0 + w.part_len, B.n);
        const uint32_t* ctx = B.ctx;
        const uint32_t shift = w.part_shift;
        const uint32_t nbin = (n_ctx + (1u << shift) - 1) >> shift;
        __syncthreads();
        for (uint32_t c = threadIdx.x; c < nbin; c += PART_THREADS) sh[c] = 0;
        __syncthreads();
        uint32_t bad = 0;
        auto count = [&](uint32_t c) {
            if (c < n_ctx) atomicAdd(&sh[c >> shift], 1u);
            else ++bad;
        };
        uint64_t i = i0;
        if ((((uintptr_t)(ctx + i0)) & 15) == 0) {
            // 16-byte loads over the aligned body (part_len is a multiple of 4)
            const uint4* v = reinterpret_cast<const uint4*>(ctx + i0);
            const uint64_t nv = (i1 - i0) / 4;
            for (uint64_t k = threadIdx.x; k < nv; k += PART_THREADS) {
                const uint4 q = ld_stream(&v[k]);
                count(q.x); count(q.y); count(q.z); count(q.w);
            }
            i = i0 + nv * 4;
        }
        for (uint64_t j = i + threadIdx.x; j < i1; j += PART_THREADS) count(ld_stream(&ctx[j]));
        if (bad) atomicAdd(&w.buf_bad[b], (unsigned long long)bad);
        __syncthreads();
        uint32_t* out = w.part_cnt + B.cnt_base + pl;
        for (uint32_t c = threadIdx.x; c < nbin; c += PART_THREADS) out[(uint64_t)c * parts] = sh[c];
    }
}


// Shared memory of k_part_scatter for up to nb bins: per-bin cursors of the
// part, the tile's per-bin counts / offsets, and the tile's records staged in
// bin order (record + bin).
// Ahead of them sits the stage of the next tile's samples (pc, ctx, count,
// stall), filled by bulk copies while the current tile is processed.
constexpr size_t PSC_STAGE_PC = 0, PSC_STAGE_CTX = PSC_TILE * 8, PSC_STAGE_CNT = PSC_TILE * 12,
                 PSC_STAGE_ST = PSC_TILE * 16, PSC_STAGE = ((size_t)PSC_TILE * 17 + 127) & ~(size_t)127;

__host__ __device__ inline size_t part_scatter_smem(uint32_t nb) {
    return PSC_STAGE + (size_t)nb * 4 + ((size_t)nb + 1) * 4 + 8 + (size_t)PSC_TILE * (8 + 2);
}

// Each part is processed in tiles of PART_TILE samples: the tile's records
// are ranked by bin with shared-memory atomics, staged in bin order, and
// then written so that consecutive threads store consecutive records of a
// bin (coalesced runs instead of lone 8-byte stores, which the L2 would have
// to merge with DRAM data when it evicts partly written sectors).  A full
// tile whose arrays are 16-byte aligned arrives by bulk copies (TMA) into the
// stage, issued by one thread as soon as every thread has read the previous
// tile from it, so the next tile's loads overlap this tile's lookups and
// stores; other tiles are loaded by the threads themselves.
template <bool HAS_CNT, int U>
__global__ void __launch_bounds__(PSC_THREADS, PSC_MIN_BLOCKS) k_part_scatter(AggWork w) {
    static_assert(PSC_TILE == PSC_THREADS * U, "one tile = U samples per thread");
    constexpr int PART_THREADS = PSC_THREADS, PART_TILE = PSC_TILE;
    extern __shared__ __align__(128) unsigned char psm[];
    __shared__ uint32_t sw[33];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t s_abort;
    const uint32_t nbmax = w.part_ctx_max;
    uint64_t* spc = reinterpret_cast<uint64_t*>(psm + PSC_STAGE_PC);
    uint32_t* sctx = reinterpret_cast<uint32_t*>(psm + PSC_STAGE_CTX);
    uint32_t* scnt = reinterpret_cast<uint32_t*>(psm + PSC_STAGE_CNT);
    uint8_t* sst = psm + PSC_STAGE_ST;
    uint32_t* cur = reinterpret_cast<uint32_t*>(psm + PSC_STAGE);      // [nbmax] cursors of the part
    uint32_t* th = cur + nbmax;                                         // [nbmax + 1] tile counts -> offsets
    uint2* srec = reinterpret_cast<uint2*>(psm + PSC_STAGE + (((size_t)nbmax * 4 + ((size_t)nbmax + 1) * 4 + 7) & ~(size_t)7));
    uint16_t* sbin = reinterpret_cast<uint16_t*>(srec + PART_TILE);
    const uint64_t keep = policy_evict_last();
    const uint64_t once = policy_evict_first();      // samples and records pass through L2 once: the tables stay
    const uint32_t limit = w.timeout_iters ? w.timeout_iters : (1u << 22);
    if (threadIdx.x == 0) { mbar_init(&bar); s_abort = 0; }
    uint32_t phase = 0;
    bool aborted = false;
    for (uint64_t p = blockIdx.x; p < w.n_parts && !aborted; p += gridDim.x) {
        const uint32_t b = upper_index<uint64_t>(w.buf_part, w.n_buf, p);
        const BufDev B = w.bufs[b];
        const DevBinary bin = w.bins[B.bin];
        const uint32_t n_ctx = B.n_ctx;
        const uint64_t pl = p - B.part_base;
        const uint64_t parts = w.buf_part[b + 1] - w.buf_part[b];
        const uint64_t i0 = pl * w.part_len, i1 = min(i0 + w.part_len, B.n);
        __syncthreads();                                // the previous part's cursors are done
        const uint32_t shift = w.part_shift, dmask = (1u << shift) - 1;
        const uint32_t nbin = (n_ctx + dmask) >> shift;
        const bool two = w.part_mode == 2;
        const uint32_t* first = w.part_cnt + B.cnt_base + pl;
        for (uint32_t c = threadIdx.x; c < nbin; c += PART_THREADS) cur[c] = first[(uint64_t)c * parts];
        const bool cnt_in = HAS_CNT && B.count;
        // a full tile whose four source ranges start on 16-byte boundaries (all
        // sizes are multiples of 16 bytes)
        auto staged = [&](uint64_t t) {
            return t + PART_TILE <= i1 && aligned16(B.pc + t) && aligned16(B.ctx + t) && aligned16(B.stall + t) &&
                   (!cnt_in || aligned16(B.count + t));
        };
        auto issue = [&](uint64_t t) {                  // one thread; every thread is done with the stage
            fence_proxy_async();
            mbar_expect_tx(&bar, PART_TILE * (cnt_in ? 8u + 4u + 1u + 4u : 8u + 4u + 1u));
            bulk_g2s_hint(spc, B.pc + t, PART_TILE * 8, &bar, once);
            bulk_g2s_hint(sctx, B.ctx + t, PART_TILE * 4, &bar, once);
            bulk_g2s_hint(sst, B.stall + t, PART_TILE, &bar, once);
            if (cnt_in) bulk_g2s_hint(scnt, B.count + t, PART_TILE * 4, &bar, once);
        };
        if (threadIdx.x == 0 && staged(i0)) issue(i0);
        uint32_t bad = 0;
        for (uint64_t t0 = i0; t0 < i1; t0 += PART_TILE) {
            for (uint32_t c = threadIdx.x; c <= nbin; c += PART_THREADS) th[c] = 0;
            const bool from_stage = staged(t0);
            if (from_stage) {
                if (!mbar_wait(&bar, phase, limit)) {
                    s_abort = 1;
                    raise_status(w.status, 7 /* HPA_E_TIMEOUT */, 1);
                }
                phase ^= 1u;
            }
            __syncthreads();
            if (s_abort) { aborted = true; break; }
            uint64_t pc[U];
            uint32_t st[U], cnt[U], cx[U], nd[U], rk[U];
            bool ok[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const uint32_t k = (uint32_t)u * PART_THREADS + threadIdx.x;
                const uint64_t i = t0 + k;
                ok[u] = i < i1;
                pc[u] = 0; st[u] = 0; cnt[u] = 1u; cx[u] = 0xFFFFFFFFu;
                if (from_stage) {
                    cx[u] = sctx[k];
                    st[u] = sst[k];
                    pc[u] = spc[k];
                    if (cnt_in) cnt[u] = scnt[k];
                    ok[u] = cx[u] < n_ctx;
                } else if (ok[u]) {
                    cx[u] = ld_stream(&B.ctx[i]);
                    st[u] = ld_stream(&B.stall[i]);
                    pc[u] = ld_stream((const unsigned long long*)&B.pc[i]);
                    if (cnt_in) cnt[u] = ld_stream(&B.count[i]);
                    ok[u] = cx[u] < n_ctx;                  // counted as invalid by k_part_hist
                }
            }
            lookup_nodes<U>(bin, pc, ok, nd, keep, w.status);
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (ok[u]) rk[u] = atomicAdd(&th[cx[u] >> shift], 1u);
            __syncthreads();
            if (threadIdx.x == 0 && staged(t0 + PART_TILE)) issue(t0 + PART_TILE);
            // one counter per thread when the bins fit (the two-level path's buckets)
            const uint32_t tot = nbin <= (uint32_t)PSC_THREADS
                                     ? block_scan_array<uint32_t, PSC_THREADS, 1>(th, (int)nbin, sw)
                                     : block_scan_array<uint32_t, PSC_THREADS, PSC_SCAN_EPT>(th, (int)nbin, sw);
            if (threadIdx.x == 0) th[nbin] = tot;
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (!ok[u]) continue;
                const bool bad_stall = st[u] >= B.n_stall;
                const uint32_t sub = bad_stall ? 0u : ((nd[u] << w.sb) | st[u]);
                const uint32_t q = th[cx[u] >> shift] + rk[u];
                if (!in_bounds(w.status, q, PART_TILE, 102)) continue;     // site 102: tile stage
                srec[q] = make_uint2(sub, bad_stall ? 0u : cnt[u]);
                sbin[q] = (uint16_t)(two ? ((cx[u] >> shift) << 8 | (cx[u] & dmask)) : cx[u]);
                bad += bad_stall;
            }
            __syncthreads();
            for (uint32_t j = threadIdx.x; j < tot; j += PART_THREADS) {
                const uint32_t sb = sbin[j];
                const uint32_t c = two ? sb >> 8 : sb;
                const uint32_t dst = cur[c] + (j - th[c]);
                if (!in_bounds(w.status, dst, w.n_rec, 103)) continue;     // site 103: record destination
                if (two) {
                    if (HAS_CNT) __stcs((unsigned long long*)&w.rec2_pair[dst], *(const unsigned long long*)&srec[j]);
                    else __stcs(&w.rec2_sub[dst], srec[j].x);
                    __stcs((signed char*)&w.rec2_dig[dst], (signed char)(uint8_t)sb);
                } else {
                    if (HAS_CNT) __stcs((unsigned long long*)&w.rec_pair[dst], *(const unsigned long long*)&srec[j]);
                    else __stcs(&w.rec_sub[dst], srec[j].x);
                }
            }
            __syncthreads();
            for (uint32_t c = threadIdx.x; c < nbin; c += PART_THREADS) cur[c] += th[c + 1] - th[c];
            __syncthreads();
        }
        if (bad) atomicAdd(&w.buf_bad[b], (unsigned long long)bad);
    }
    // after a wait gave up, the copies of that tile may still be in flight:
    // wait for them (bounded again, by at least 2^22 polls whatever the
    // option says) before the CTA's shared memory goes away
    if (aborted) mbar_wait(&bar, phase ^ 1u, max(limit, 1u << 22));
}

// ------------------------------------------------------------------ second pass (part_mode 2)
// Segment s = (buffer b, bucket k): the records of contexts [k << shift,
// (k + 1) << shift) of b, contiguous in the second record buffer after the
// first pass.  Each segment is cut into chunks of PART2_LEN records; the
// counters of chunk j of segment s for digit d (a context's low bits) sit at
// cnt2[(seg_chunk[s] << shift) + d * chunks(s) + j], digit-major within the
// segment, so one exclusive scan places every (context, chunk).
__device__ __forceinline__ void seg_bounds(const AggWork& w, uint32_t s, uint64_t& start, uint64_t& end) {
    const uint32_t b = upper_index<uint32_t>(w.buf_seg, w.n_buf, s);
    const BufDev& B = w.bufs[b];
    const uint64_t parts = w.buf_part[b + 1] - w.buf_part[b];
    const uint64_t k = s - B.seg_base;
    start = w.part_cnt[B.cnt_base + k * parts];
    end = w.part_cnt[B.cnt_base + (k + 1) * parts];     // the next bucket's start, or the next buffer's
}

__global__ void k_seg_chunks(AggWork w) {
    for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < w.n_seg; s += gridDim.x * blockDim.x) {
        uint64_t a, e;
        seg_bounds(w, s, a, e);
        w.seg_chunk[s] = (uint32_t)((e - a + PART2_LEN - 1) / PART2_LEN);
    }
}

// chunk k -> segment s, chunk j within it, its record range and chunk count
__device__ __forceinline__ void chunk_of(const AggWork& w, uint32_t k, uint32_t& s, uint32_t& j, uint32_t& chs,
                                         uint64_t& a, uint64_t& e) {
    s = upper_index<uint32_t>(w.seg_chunk, w.n_seg, k);
    j = k - w.seg_chunk[s];
    chs = w.seg_chunk[s + 1] - w.seg_chunk[s];
    uint64_t sa, se;
    seg_bounds(w, s, sa, se);
    a = sa + (uint64_t)j * PART2_LEN;
    e = min(a + PART2_LEN, se);
}

__global__ void __launch_bounds__(PART_THREADS) k_part2_hist(AggWork w) {
    __shared__ uint32_t h[256];
    const uint32_t n_chunks = w.seg_chunk[w.n_seg];
    const uint32_t nd = 1u << w.part_shift;
    for (uint32_t k = blockIdx.x; k < n_chunks; k += gridDim.x) {
        uint32_t s, j, chs;
        uint64_t a, e;
        chunk_of(w, k, s, j, chs, a, e);
        __syncthreads();
        for (uint32_t d = threadIdx.x; d < nd; d += PART_THREADS) h[d] = 0;
        __syncthreads();
        for (uint64_t i = a + threadIdx.x; i < e; i += PART_THREADS) atomicAdd(&h[w.rec2_dig[i]], 1u);
        __syncthreads();
        uint32_t* out = w.cnt2 + ((uint64_t)w.seg_chunk[s] << w.part_shift) + j;
        for (uint32_t d = threadIdx.x; d < nd; d += PART_THREADS) out[(uint64_t)d * chs] = h[d];
    }
}

// group offsets (exclusive) from the scanned second-pass counters
__global__ void k_part2_seg(AggWork w) {
    for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g <= w.G; g += gridDim.x * blockDim.x) {
        if (g == w.G) { w.grp_hist[g] = w.cnt2[w.n_cnt2]; continue; }
        const uint32_t b = upper_index<uint32_t>(w.buf_grp, w.n_buf, g);
        const BufDev& B = w.bufs[b];
        const uint32_t c = g - B.grp_base;
        const uint32_t s = B.seg_base + (c >> w.part_shift);
        const uint32_t d = c & ((1u << w.part_shift) - 1);
        const uint32_t chs = w.seg_chunk[s + 1] - w.seg_chunk[s];
        w.grp_hist[g] = w.cnt2[((uint64_t)w.seg_chunk[s] << w.part_shift) + (uint64_t)d * chs];
    }
}

// second pass: each chunk's records staged by digit, tile by tile, and
// written as coalesced runs to their contexts' segments
template <bool HAS_CNT>
__global__ void __launch_bounds__(PART_THREADS, 2) k_part2_scatter(AggWork w) {
    constexpr int U = PART_U;
    __shared__ uint32_t cur[256], th[257], sw[33];
    __shared__ uint2 srec[PART_TILE];
    __shared__ uint8_t sdig[PART_TILE];
    const uint32_t n_chunks = w.seg_chunk[w.n_seg];
    const uint32_t nd = 1u << w.part_shift;
    for (uint32_t k = blockIdx.x; k < n_chunks; k += gridDim.x) {
        uint32_t s, j, chs;
        uint64_t a, e;
        chunk_of(w, k, s, j, chs, a, e);
        __syncthreads();
        const uint32_t* first = w.cnt2 + ((uint64_t)w.seg_chunk[s] << w.part_shift) + j;
        for (uint32_t d = threadIdx.x; d < nd; d += PART_THREADS) cur[d] = first[(uint64_t)d * chs];
        for (uint64_t t0 = a; t0 < e; t0 += PART_TILE) {
            for (uint32_t d = threadIdx.x; d <= nd; d += PART_THREADS) th[d] = 0;
            __syncthreads();
            uint2 r[U];
            uint32_t dg[U], rk[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const uint64_t i = t0 + (uint64_t)u * PART_THREADS + threadIdx.x;
                dg[u] = 0xFFFFFFFFu;
                if (i < e) {
                    if (HAS_CNT) r[u] = ld_stream(&w.rec2_pair[i]);
                    else r[u].x = ld_stream(&w.rec2_sub[i]);
                    dg[u] = w.rec2_dig[i];
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (dg[u] != 0xFFFFFFFFu) rk[u] = atomicAdd(&th[dg[u]], 1u);
            __syncthreads();
            const uint32_t tot = block_scan_array<uint32_t, PART_THREADS, 1>(th, (int)nd, sw);
            if (threadIdx.x == 0) th[nd] = tot;
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (dg[u] == 0xFFFFFFFFu) continue;
                const uint32_t q = th[dg[u]] + rk[u];
                if (!in_bounds(w.status, q, PART_TILE, 104)) continue;     // site 104: tile stage
                srec[q] = r[u];
                sdig[q] = (uint8_t)dg[u];
            }
            __syncthreads();
            for (uint32_t i = threadIdx.x; i < tot; i += PART_THREADS) {
                const uint32_t d = sdig[i];
                const uint32_t dst = cur[d] + (i - th[d]);
                if (!in_bounds(w.status, dst, w.n_rec, 105)) continue;     // site 105: record destination
                if (HAS_CNT) __stcs((unsigned long long*)&w.rec_pair[dst], *(const unsigned long long*)&srec[i]);
                else __stcs(&w.rec_sub[dst], srec[i].x);
            }
            __syncthreads();
            for (uint32_t d = threadIdx.x; d < nd; d += PART_THREADS) cur[d] += th[d + 1] - th[d];
            __syncthreads();
        }
    }
}

// ------------------------------------------------------------------ K10: split big groups
// One CTA per big group: fine-bin histogram, offsets, leaf boundaries (runs
// of bins, see big_leaf_head) and a scatter by bin into rec2 (the order
// within a bin is free: its leaf sorts it).  Both passes load BIG_U records
// per thread before their shared-memory atomics, to keep loads in flight.
// (Warp-aggregating those atomics with __match_any_sync made the pass 2.6x
// slower: hot bins are not what limits it.)
constexpr int BIG_U = 4;

__global__ void __launch_bounds__(BIG_THREADS, 2) k_big_partition(AggWork w) {
    extern __shared__ uint32_t off[];            // 2^h + 1 bin counts, then offsets, then cursors
    __shared__ uint32_t sw[33];
    const uint32_t n_items = w.item_id[w.G];
    const uint32_t* seg = w.grp_hist;
    const uint32_t* leaf_base = w.item_nleaf;
    const uint32_t q = w.q;
    const uint32_t h = fine_bits(w.sbits), nb = 1u << h, shift = w.sbits - h;
    const bool pair = w.rec_pair != nullptr;
    for (uint32_t it = blockIdx.x; it < n_items; it += gridDim.x) {
        const uint32_t g0 = w.item_grp0[it];
        const uint32_t g1 = (it + 1 < n_items) ? w.item_grp0[it + 1] : w.G;
        const uint32_t s0 = seg[g0], s1 = seg[g1];
        const uint32_t n = s1 - s0;
        if (n <= w.cap) continue;                 // uniform across the block
        for (uint32_t j = threadIdx.x; j <= nb; j += BIG_THREADS) off[j] = 0;
        __syncthreads();
        for (uint32_t i0 = s0 + threadIdx.x; i0 < s1; i0 += BIG_THREADS * BIG_U) {
            uint32_t k[BIG_U];
#pragma unroll
            for (int u = 0; u < BIG_U; ++u) {
                const uint32_t i = i0 + u * BIG_THREADS;
                if (i < s1) k[u] = pair ? w.rec_pair[i].x : w.rec_sub[i];
            }
#pragma unroll
            for (int u = 0; u < BIG_U; ++u)
                if (i0 + u * BIG_THREADS < s1) atomicAdd(&off[k[u] >> shift], 1u);
        }
        __syncthreads();
        block_scan_array<uint32_t, BIG_THREADS, BIG_EPT>(off, nb + 1, sw);   // off[nb] = n
        // leaf boundaries
        const uint32_t slots = big_leaf_slots(n, q);
        const uint32_t l0 = leaf_base[it];
        const uint32_t b = upper_index<uint32_t>(w.buf_grp, w.n_buf, g0);
        const uint32_t j0 = threadIdx.x * BIG_EPT;
        uint32_t c = 0;
#pragma unroll 4
        for (uint32_t k = 0; k < BIG_EPT; ++k)
            if (j0 + k < nb) c += big_leaf_head(off, j0 + k, q);
        uint32_t n_lv;
        uint32_t at = block_exclusive_scan<uint32_t, BIG_THREADS>(c, sw, &n_lv);
        for (uint32_t k = 0; k < BIG_EPT && c; ++k) {
            const uint32_t j = j0 + k;
            if (j < nb && big_leaf_head(off, j, q)) {
                if (at < slots) w.leaf_start[l0 + at] = s0 + off[j];
                ++at;
                --c;
            }
        }
        if (n_lv > slots && threadIdx.x == 0) raise_status(w.status, 8 /* HPA_E_INTERNAL */, 10);
        __syncthreads();
        const uint32_t nl = min(n_lv, slots);
        for (uint32_t k = threadIdx.x; k < slots; k += BIG_THREADS) {
            if (k >= nl) w.leaf_start[l0 + k] = s1;   // unused slot: empty leaf
            w.leaf_end[l0 + k] = (k + 1 < nl) ? w.leaf_start[l0 + k + 1] : s1;
            w.leaf_grp0[l0 + k] = g0;
            w.leaf_info[l0 + k] = (b << 8) | 1u;
        }
        __syncthreads();
        for (uint32_t i0 = s0 + threadIdx.x; i0 < s1; i0 += BIG_THREADS * BIG_U) {
            uint2 r[BIG_U];
#pragma unroll
            for (int u = 0; u < BIG_U; ++u) {
                const uint32_t i = i0 + u * BIG_THREADS;
                if (i < s1) {
                    if (pair) r[u] = w.rec_pair[i];
                    else r[u].x = w.rec_sub[i];
                }
            }
#pragma unroll
            for (int u = 0; u < BIG_U; ++u) {
                const uint32_t i = i0 + u * BIG_THREADS;
                if (i >= s1) break;
                const uint32_t p = s0 + atomicAdd(&off[r[u].x >> shift], 1u);
                if (!in_bounds(w.status, p, s1, 106)) continue;              // site 106: big-group record
                if (pair) {
                    w.rec2_pair[p] = r[u];
                } else {
                    w.rec2_sub[p] = r[u].x;
                    if (w.val64) w.rec2_v64[p] = w.rec_v64[i];
                }
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ K13: emit
// Leaves are in key order, so leaf_out (the scanned run counts) places every
// key (of every leaf, or with fused leaves of those that left their keys in
// tmp_key / tmp_val).  With emit_totals, the per-stall totals and UNKNOWN totals of each
// buffer are summed here over its keys (every valid record lies in exactly
// one key): per-thread slots in shared memory, flushed when the CTA moves to
// another buffer.
constexpr int EMIT_U = 4;

__global__ void __launch_bounds__(256) k_emit(AggWork w) {
    extern __shared__ unsigned long long acc[];          // [2^sb][256] per-thread totals (emit_totals)
    __shared__ unsigned long long unk[HPA_MAX_STALL_DEV];
    const uint32_t tid = threadIdx.x;
    const uint32_t n_leaves = w.item_nleaf[w.G];
    const uint32_t* leaf_out = w.leaf_d;
    const uint32_t smask = (w.sbits >= 32) ? 0xFFFFFFFFu : ((1u << w.sbits) - 1);
    const uint32_t stmask = (1u << w.sb) - 1;
    const uint32_t nsm = 1u << w.sb;
    const bool tot = w.emit_totals != 0;
    if (tot) {
        for (uint32_t r = 0; r < nsm; ++r) acc[r * 256 + tid] = 0;
        if (tid < HPA_MAX_STALL_DEV) unk[tid] = 0;
    }
    __syncthreads();
    uint32_t cur_b = 0xFFFFFFFFu;
    auto flush = [&]() {
        __syncthreads();
        if (cur_b != 0xFFFFFFFFu) {
            const BufDev& B = w.bufs[cur_b];
            for (uint32_t r = tid >> 5; r < nsm; r += 8) {
                unsigned long long v = 0;
                for (uint32_t t = lane_id(); t < 256; t += 32) { v += acc[r * 256 + t]; acc[r * 256 + t] = 0; }
                v = warp_sum(v);
                if (lane_id() == 0 && v && B.total) atomicAdd((unsigned long long*)&B.total[r], v);
                if (lane_id() == 0 && unk[r] && B.unknown) atomicAdd((unsigned long long*)&B.unknown[r], unk[r]);
            }
        }
        __syncthreads();
        if (tid < HPA_MAX_STALL_DEV) unk[tid] = 0;
        __syncthreads();
    };
    for (uint32_t l = blockIdx.x; l < n_leaves; l += gridDim.x) {
        const uint32_t d = leaf_out[l + 1] - leaf_out[l];
        if (d == 0) continue;                             // uniform across the block
        if (w.fuse_emit && (w.leaf_look[l] & LOOK_DIRECT)) continue;   // the leaf wrote its keys itself
        const uint32_t info = w.leaf_info[l];
        const uint32_t b = info >> 8;
        const BufDev& B = w.bufs[b];
        if (w.buf_bad[b]) continue;
        if (tot && b != cur_b) { flush(); cur_b = b; }
        const uint32_t M = w.bins[B.bin].n_nodes;
        const uint32_t start = w.leaf_start[l];
        const uint32_t g0 = w.leaf_grp0[l];
        const uint64_t o0 = (uint64_t)leaf_out[l] - leaf_out[w.buf_first_leaf[b]];
        const uint32_t gctx0 = g0 - B.grp_base;
        // EMIT_U keys per thread loaded before any is processed: more bytes in flight
        for (uint32_t i0 = tid; i0 < d; i0 += EMIT_U * 256) {
            uint32_t kk[EMIT_U];
            unsigned long long vv[EMIT_U];
#pragma unroll
            for (int u = 0; u < EMIT_U; ++u) {
                const uint32_t i = i0 + u * 256;
                if (i < d) {
                    if (in_bounds(w.status, (uint64_t)start + i, w.n_rec, 110)) {   // site 110: leaf key
                        kk[u] = __ldcs(&w.tmp_key[start + i]);
                        vv[u] = __ldcs((const unsigned long long*)&w.tmp_val[start + i]);
                    } else {
                        kk[u] = 0;
                        vv[u] = 0;
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < EMIT_U; ++u) {
                const uint32_t i = i0 + u * 256;
                if (i >= d) break;
                const uint64_t pos = o0 + i;
                const uint32_t k = kk[u];
                const unsigned long long v = vv[u];
                const uint32_t sub = k & smask;
                const uint32_t node = sub >> w.sb;
                const uint32_t stall = sub & stmask;
                if (tot) {
                    acc[stall * 256 + tid] += v;
                    if (node == M) atomicAdd(&unk[stall], v);
                }
                if (pos < B.capacity) {
                    const uint32_t gl = (w.sbits >= 32) ? 0u : (k >> w.sbits);
                    __stcs(&B.key_ctx[pos], gctx0 + gl);
                    __stcs(&B.key_node[pos], (node == M) ? UNKNOWN : node);
                    B.key_stall[pos] = (uint8_t)stall;
                    __stcs((unsigned long long*)&B.val[pos], v);
                }
            }
        }
    }
    if (tot) flush();
}

// per-buffer key counts and status, from the scanned leaf key counts (doing
// this in k_emit's first CTA instead of a launch of its own made k_emit 0.47
// ms slower on the large profile)
__device__ __forceinline__ void finalize_range(const AggWork& w, uint32_t i0, uint32_t step) {
    const uint32_t* leaf_out = w.leaf_d;
    for (uint32_t b = i0; b < w.n_buf; b += step) {
        const BufDev& B = w.bufs[b];
        const uint64_t K = (uint64_t)leaf_out[w.buf_first_leaf[b + 1]] - leaf_out[w.buf_first_leaf[b]];
        const unsigned long long bad = w.buf_bad[b];
        if (bad) {
            *B.n_keys = 0;
            atomicAdd(&w.status->bad, bad);
            raise_status(w.status, 3 /* HPA_E_INVALID_SAMPLE */, (int32_t)b);
        } else {
            *B.n_keys = K;
            if (K > B.capacity) raise_status(w.status, 4 /* HPA_E_CAPACITY */, (int32_t)b);
        }
    }
}

__global__ void k_finalize(AggWork w) { finalize_range(w, threadIdx.x, blockDim.x); }

// ------------------------------------------------------------------ driver
// seg_ready: the group offsets are in grp_hist already; part_seg: they come
// from the scanned part counts (partition path, part_mode 1)
void run_plan(const AggWork& w, cudaStream_t s, int sms, uint64_t* launches, bool seg_ready, bool part_seg) {
    const int gblocks = (int)std::max<uint64_t>(1, std::min<uint64_t>((w.G + 256) / 256, (uint64_t)sms * 16));
    if (w.G <= PLAN_ONE_CTA_MAX) {
        k_plan_one<<<1, SCAN_SMALL_THREADS, 0, s>>>(w, part_seg ? 1 : (seg_ready ? 2 : 0));
        *launches += 1;
        return;
    }
    if (part_seg) {
        k_part_seg<<<gblocks, 256, 0, s>>>(w);
        *launches += 1;
    } else if (!seg_ready) {
        scan_u32(w.grp_hist, w.grp_hist, w.G, w.scan_tmp, s, launches);
    }
    k_item_flags<<<gblocks, 256, 0, s>>>(w);
    scan_u32(w.item_id, w.item_id, w.G, w.scan_tmp, s, launches);
    k_items<<<gblocks, 256, 0, s>>>(w);
    k_items_size<<<gblocks, 256, 0, s>>>(w);
    scan_u32(w.item_nleaf, w.item_nleaf, w.G, w.scan_tmp, s, launches);
    k_leaves<<<gblocks, 256, 0, s>>>(w);
    *launches += 4;
}

void launch_finalize(const AggWork& w, cudaStream_t s, uint64_t* launches) {
    k_finalize<<<1, 256, 0, s>>>(w);
    *launches += 1;
}

void launch_big_partition(const AggWork& w, cudaStream_t s, int sms, uint64_t* launches) {
    constexpr size_t smem = ((1u << BIG_FINE_MAX_LOG) + 1) * 4;
    set_smem_limit((const void*)k_big_partition, (int)smem);
    k_big_partition<<<sms * 3, BIG_THREADS, smem, s>>>(w);
    *launches += 1;
}

// Leaves write the final keys themselves (fused) when one leaf kernel takes
// every leaf of the call and the records carry 32-bit counts or none;
// otherwise they leave their keys in tmp_key / tmp_val for k_emit.
static bool can_fuse(const AggWork& w) {
    return w.leaf_look && w.leaf_ticket && !w.val64 && !w.small_leaves && !w.emit_separate;
}

static void run_finish(const AggWork& w_in, cudaStream_t s, int sms, uint64_t* launches, cudaEvent_t* ev) {
    AggWork w = w_in;
    w.fuse_emit = can_fuse(w) ? 1u : 0u;
    launch_big_partition(w, s, sms, launches);
    if (ev) cudaEventRecord(ev[3], s);
    launch_leaves(w, s, sms, launches);
    if (ev) cudaEventRecord(ev[4], s);
    scan_u32(w.leaf_d, w.leaf_d, w.L_max, w.scan_tmp, s, launches);
    // keys left in tmp_key / tmp_val (every leaf, or the fused leaves that
    // did not wait for their offset) are placed by k_emit
    const size_t emit_smem = w.emit_totals ? ((size_t)256 << w.sb) * 8 : 0;
    set_smem_limit((const void*)k_emit, 256 * HPA_MAX_STALL_DEV * 8);
    // leaves in small portions: up to 128 CTAs per SM, never more than the leaf
    // table's size (on the large profile 128 per SM took 0.983 ms, 64 1.005, 32
    // 1.056, 16 1.14, 8 1.19)
    const int eg = (int)std::max<uint64_t>((uint64_t)sms * 8, std::min<uint64_t>((uint64_t)sms * 128, w.L_max));
    k_emit<<<eg, 256, emit_smem, s>>>(w);
    *launches += 1;
    launch_finalize(w, s, launches);
    if (ev) cudaEventRecord(ev[5], s);
}

// One launch zeroes the per-call counters of the work area (and, with
// totals, the buffers' per-stall and UNKNOWN totals), where five memsets and
// a kernel were six graph nodes.
__global__ void k_clear(AggWork w, int totals) {
    const uint64_t nh = (uint64_t)w.G + 1, nd = (uint64_t)w.L_max + 1, nb = w.n_buf;
    const uint64_t nl = w.leaf_look ? w.L_max : 0, nt = w.leaf_ticket ? 1 : 0;
    const uint64_t n = nh + nd + nb + nl + nt;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t j = i;
        if (j < nh) { w.grp_hist[j] = 0; continue; }
        j -= nh;
        if (j < nd) { w.leaf_d[j] = 0; continue; }
        j -= nd;
        if (j < nb) { w.buf_bad[j] = 0; continue; }
        j -= nb;
        if (j < nl) { w.leaf_look[j] = 0; continue; }
        *w.leaf_ticket = 0;
    }
    if (totals)
        for (uint32_t b = blockIdx.x; b < w.n_buf; b += gridDim.x) {
            const BufDev& B = w.bufs[b];
            for (uint32_t r = threadIdx.x; r < B.n_stall; r += blockDim.x) {
                if (B.total) B.total[r] = 0;
                if (B.unknown) B.unknown[r] = 0;
            }
        }
}

void clear_work(const AggWork& w, cudaStream_t s, bool totals) {
    const uint64_t n = (uint64_t)w.G + w.L_max + w.n_buf + w.L_max + 3;
    const int blocks = (int)std::max<uint64_t>(std::min<uint64_t>(w.n_buf, 1024),
                                               std::min<uint64_t>((n + 255) / 256, 1024));
    k_clear<<<blocks, 256, 0, s>>>(w, totals ? 1 : 0);
}

void run_aggregate(const AggWork& w, cudaStream_t s, int sms, uint64_t* launches, cudaEvent_t* ev) {
    if (ev) cudaEventRecord(ev[0], s);
    clear_work(w, s, true);
    if (w.part_mode) {
        const size_t csm = (size_t)w.part_ctx_max * 4;
        const size_t ssm = part_scatter_smem(w.part_ctx_max);
        {
            const int mx = (int)PART_CTX_MAX * 4, mxs = (int)part_scatter_smem(PART_CTX_MAX);
            set_smem_limit((const void*)k_part_hist, mx);
            set_smem_limit((const void*)k_part_scatter<true, PSC_U>, mxs);
            set_smem_limit((const void*)k_part_scatter<false, PSC_U>, mxs);
        }
        // up to 8 histogram CTAs per SM, one part each (2 per SM: 0.09 ms more on the large profile)
        const int pb = (int)std::max<uint64_t>(1, std::min<uint64_t>(w.n_parts, (uint64_t)sms * 8));
        const int psb = (int)std::max<uint64_t>(1, std::min<uint64_t>(w.n_parts, (uint64_t)sms * PSC_MIN_BLOCKS));
        k_part_hist<<<pb, PART_THREADS, csm, s>>>(w);
        scan_u32(w.part_cnt, w.part_cnt, w.n_cnt, w.scan_tmp, s, launches);
        *launches += 1;
        if (w.part_mode == 1) {
            run_plan(w, s, sms, launches, true, true);
            if (ev) cudaEventRecord(ev[1], s);
            if (w.has_cnt) k_part_scatter<true, PSC_U><<<psb, PSC_THREADS, ssm, s>>>(w);
            else k_part_scatter<false, PSC_U><<<psb, PSC_THREADS, ssm, s>>>(w);
            *launches += 1;
        } else {
            // first pass into buckets, then each bucket by context
            if (ev) cudaEventRecord(ev[1], s);
            if (w.has_cnt) k_part_scatter<true, PSC_U><<<psb, PSC_THREADS, ssm, s>>>(w);
            else k_part_scatter<false, PSC_U><<<psb, PSC_THREADS, ssm, s>>>(w);
            const int sg = (int)std::max<uint64_t>(1, std::min<uint64_t>((w.n_seg + 255) / 256, (uint64_t)sms * 4));
            k_seg_chunks<<<sg, 256, 0, s>>>(w);
            scan_u32(w.seg_chunk, w.seg_chunk, w.n_seg, w.scan_tmp, s, launches);
            cudaMemsetAsync(w.cnt2, 0, sizeof(uint32_t) * ((size_t)w.n_cnt2 + 1), s);
            k_part2_hist<<<sms * 4, PART_THREADS, 0, s>>>(w);
            scan_u32(w.cnt2, w.cnt2, w.n_cnt2, w.scan_tmp, s, launches);
            const int gb = (int)std::max<uint64_t>(1, std::min<uint64_t>((w.G + 256) / 256, (uint64_t)sms * 16));
            k_part2_seg<<<gb, 256, 0, s>>>(w);
            run_plan(w, s, sms, launches, true);
            if (w.has_cnt) k_part2_scatter<true><<<sms * 2, PART_THREADS, 0, s>>>(w);
            else k_part2_scatter<false><<<sms * 2, PART_THREADS, 0, s>>>(w);
            *launches += 5;
        }
    } else {
        const size_t hsm = (size_t)HIST_SMEM_MAX * 4;
        const int per_sm = 2;
        const int hist_blocks = (int)std::max<uint64_t>(1, std::min<uint64_t>(w.n_tiles, (uint64_t)sms * per_sm));
        set_smem_limit((const void*)k_grp_hist, (int)hsm);
        k_grp_hist<<<hist_blocks, 256, hsm, s>>>(w);
        *launches += 1;
        run_plan(w, s, sms, launches, false);
        if (ev) cudaEventRecord(ev[1], s);
        const int at_blocks = (int)std::max<uint64_t>(1, std::min<uint64_t>(w.n_tiles, (uint64_t)sms * 4));
        const int sc_blocks = (int)std::max<uint64_t>(1, std::min<uint64_t>(w.n_tiles, (uint64_t)sms * 8));
        if (w.has_cnt) {
            k_attribute<true, 4><<<at_blocks, 256, 0, s>>>(w);
            k_scatter<true, 8><<<sc_blocks, 256, 0, s>>>(w);
        } else {
            k_attribute<false, 4><<<at_blocks, 256, 0, s>>>(w);
            k_scatter<false, 8><<<sc_blocks, 256, 0, s>>>(w);
        }
        *launches += 2;
    }
    if (ev) cudaEventRecord(ev[2], s);
    run_finish(w, s, sms, launches, ev);
}

// ------------------------------------------------------------------ inclusive over the structure tree
// (Section 6.1: values propagate up the tree).  Each key is expanded to its
// node and every ancestor up to the function node, then the expanded records
// are aggregated by the same plan / leaf / emit kernels with 64-bit values.
__global__ void k_expand_hist(AggWork w, ExpandSrc x) {
    const uint64_t K = min(*x.n_keys, x.cap);
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < K; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t c = x.ctx[i], n = x.node[i];
        if (c >= x.n_ctx || (n != UNKNOWN && n >= x.M)) { atomicAdd(&w.buf_bad[0], 1ull); continue; }
        atomicAdd(&w.grp_hist[c], n == UNKNOWN ? 1u : x.depth[n] + 1u);
    }
}

__global__ void k_expand_scatter(AggWork w, ExpandSrc x) {
    const uint64_t K = min(*x.n_keys, x.cap);
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < K; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t c = x.ctx[i], n0 = x.node[i];
        if (c >= x.n_ctx || (n0 != UNKNOWN && n0 >= x.M)) continue;
        const uint32_t r = x.stall[i];
        const uint64_t v = x.val[i];
        const uint32_t cnt = n0 == UNKNOWN ? 1u : x.depth[n0] + 1u;
        uint32_t slot = atomicAdd(&w.grp_cursor[(size_t)c << w.cur_shift], cnt);
        if (n0 == UNKNOWN) {
            w.rec_sub[slot] = (x.M << w.sb) | r;
            w.rec_v64[slot] = v;
            continue;
        }
        uint32_t n = n0;
        for (uint32_t k = 0; k < cnt; ++k) {
            w.rec_sub[slot + k] = (n << w.sb) | r;
            w.rec_v64[slot + k] = v;
            n = x.parent[n];
        }
    }
}

void run_group_tail(const AggWork& w, cudaStream_t s, int sms, uint64_t* launches) {
    run_finish(w, s, sms, launches, nullptr);
}

void run_expand_aggregate(const AggWork& w, const ExpandSrc& x, cudaStream_t s, int sms, uint64_t* launches) {
    clear_work(w, s);
    const int blocks = (int)std::max<uint64_t>(1, std::min<uint64_t>((x.cap + 255) / 256, (uint64_t)sms * 8));
    k_expand_hist<<<blocks, 256, 0, s>>>(w, x);
    run_plan(w, s, sms, launches, false);
    k_expand_scatter<<<blocks, 256, 0, s>>>(w, x);
    *launches += 2;
    run_finish(w, s, sms, launches, nullptr);
}

}  // namespace hpa
