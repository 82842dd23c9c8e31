// Device-side helpers shared by the hpa kernels (sm_103a).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace hpa {

constexpr uint32_t UNKNOWN = 0xFFFFFFFFu;
constexpr uint32_t NO_PARENT = 0xFFFFFFFFu;
constexpr uint32_t EMPTY_KEY = 0xFFFFFFFFu;

// Device status word of a handle.  Kernels only ever raise it (atomicCAS from
// 0), the host reads and clears it in hpa_sync.
struct DevStatus {
    int32_t code;           // first hpa_status raised by a kernel
    int32_t where;          // kernel-specific detail (which wait gave up, ...)
    unsigned long long bad; // invalid sample records
};

__device__ __forceinline__ void raise_status(DevStatus* st, int32_t code, int32_t where = 0) {
    if (atomicCAS(&st->code, 0, code) == 0) st->where = where;
}

// Bounds-checked build (compiled with -DHPA_CHECKED): an index that a kernel
// computes from counters, scans or data is checked against the size of the
// array it indexes before the access; out of range, the caller skips the
// access and the status records HPA_E_INTERNAL with `where` = the site's
// number (100 + n, listed where each check stands) -- never a trap.  In the
// normal build the check is the constant true and compiles away.
__device__ __forceinline__ bool in_bounds(DevStatus* st, uint64_t i, uint64_t n, int32_t site) {
#ifdef HPA_CHECKED
    if (i < n) return true;
    if (st) raise_status(st, 8 /* HPA_E_INTERNAL */, site);
    return false;
#else
    (void)st; (void)i; (void)n; (void)site;
    return true;
#endif
}

// Program structure of one binary as the attribution kernels read it.
//   ent[j] = {lo_j, node_j} (offsets from pc_base): entry j covers
//     [lo_j, lo_{j+1}); the ranges in order, a gap between two ranges as an
//     entry of node n_nodes (UNKNOWN), and a last entry at `span` that only
//     ends the one before it.  8 bytes per entry, so that the table stays in L2.
//   dir[b], for the bucket [b << dshift, (b + 1) << dshift) of offsets: the
//     node of the one entry that covers the whole bucket, or DIR_SEARCH | j
//     with j the entry that holds the bucket's start.
// A PC p belongs to range i iff lo_i <= p < hi_i (half-open); the entries
// tile [0, span), so p lies in exactly one of them.
constexpr uint32_t DIR_SEARCH = 0x80000000u;
constexpr uint64_t DIR_MAX_ENTRIES = 8ull << 20;    // 32 MB directory at most
constexpr uint64_t DIR_PER_ENTRY = 4;               // directory buckets per table entry, at most
constexpr uint64_t DIR_MIN_ENTRIES = 1ull << 20;    // small binaries still get 2^20 buckets

struct DevBinary {
    uint64_t pc_base;
    uint64_t span;          // range_hi[R-1] - pc_base (< 2^32)
    uint32_t dshift;
    uint32_t n_dir;
    uint32_t n_ent;         // table entries, the last one at span
    uint32_t n_nodes;       // M: UNKNOWN is coded as node M inside subkeys
    const uint32_t* dir;
    const uint2* ent;
};

// asynchronous global -> shared copies (cp.async, sm_80+)
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_all;" ::: "memory");
}

// L2 cache policies: tables that every sample probes should stay in L2
// (evict_last); data read or written once streams through (evict_first).
__device__ __forceinline__ uint64_t policy_evict_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint32_t ld_keep(const uint32_t* a, uint64_t pol) {
    uint32_t v;
    asm volatile("ld.global.nc.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(v) : "l"(a), "l"(pol));
    return v;
}
__device__ __forceinline__ uint2 ld_keep2(const uint2* a, uint64_t pol) {
    uint2 v;
    asm volatile("ld.global.nc.L2::cache_hint.v2.u32 {%0, %1}, [%2], %3;" : "=r"(v.x), "=r"(v.y) : "l"(a), "l"(pol));
    return v;
}
template <typename T>
__device__ __forceinline__ T ld_stream(const T* a) { return __ldcs(a); }
__device__ __forceinline__ void st_stream(uint2* a, uint2 v) { __stcs(a, v); }
__device__ __forceinline__ void st_stream(uint32_t* a, uint32_t v) { __stcs(a, v); }

// release / acquire accesses at GPU scope (look-back words between CTAs)
__device__ __forceinline__ void st_release_u64(unsigned long long* a, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(a), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* a) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(a) : "memory");
    return v;
}

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31; }
__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

template <typename T>
__device__ __forceinline__ T warp_inclusive_scan(T x) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if ((int)lane_id() >= o) x += y;
    }
    return x;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Block-wide exclusive scan of one value per thread.  `sw` holds >= 33
// entries of shared scratch.  Returns the exclusive prefix; *total gets the sum.
template <typename T, int THREADS>
__device__ __forceinline__ T block_exclusive_scan(T x, T* sw, T* total) {
    constexpr int W = THREADS / 32;
    const int warp = threadIdx.x >> 5;
    T inc = warp_inclusive_scan(x);
    if (lane_id() == 31) sw[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        T v = (int)lane_id() < W ? sw[lane_id()] : T(0);
        T vi = warp_inclusive_scan(v);
        if ((int)lane_id() < W) sw[lane_id()] = vi - v;
        if (lane_id() == W - 1) sw[32] = vi;
    }
    __syncthreads();
    T r = sw[warp] + inc - x;
    *total = sw[32];
    __syncthreads();
    return r;
}

// Exclusive scan, in place, of n <= THREADS * EPT values held in shared
// memory; each thread owns EPT consecutive entries.  Returns the total.
template <typename T, int THREADS, int EPT>
__device__ __forceinline__ T block_scan_array(T* a, int n, T* sw) {
    const int base = threadIdx.x * EPT;
    T loc[EPT];
    T s = 0;
#pragma unroll
    for (int i = 0; i < EPT; ++i) {
        loc[i] = (base + i < n) ? a[base + i] : T(0);
        s += loc[i];
    }
    T tot;
    T pre = block_exclusive_scan<T, THREADS>(s, sw, &tot);
#pragma unroll
    for (int i = 0; i < EPT; ++i) {
        if (base + i < n) a[base + i] = pre;
        pre += loc[i];
    }
    __syncthreads();
    return tot;
}

__host__ __device__ inline uint32_t ceil_log2_u64(uint64_t x) {
    uint32_t b = 0;
    while ((1ull << b) < x) ++b;
    return b;
}

// Exclusive scan, in place, of n counters in shared memory, walked by each
// warp over a contiguous chunk 32 entries per row (lane l reads entry
// row * 32 + l: no bank conflicts), then offset by the warps before it.
// `sw` holds >= 33 words.  Every thread of the block must call it.
template <int THREADS>
__device__ __forceinline__ void block_scan_rows(uint32_t* a, int n, uint32_t* sw) {
    constexpr int W = THREADS / 32;
    const int warp = threadIdx.x >> 5, lane = lane_id();
    const int per = max(32, ((n + W - 1) / W + 31) & ~31);
    const int a0 = min(n, warp * per), a1 = min(n, a0 + per);
    uint32_t carry = 0;
    for (int base = a0; base < a1; base += 32) {
        const int i = base + lane;
        const uint32_t v = i < a1 ? a[i] : 0u;
        const uint32_t inc = warp_inclusive_scan(v);
        if (i < a1) a[i] = carry + inc - v;
        carry += __shfl_sync(0xffffffffu, inc, 31);
    }
    if (lane == 0) sw[warp] = carry;
    __syncthreads();
    if (warp == 0) {
        const uint32_t v = lane < W ? sw[lane] : 0u;
        const uint32_t inc = warp_inclusive_scan(v);
        if (lane < W) sw[lane] = inc - v;
    }
    __syncthreads();
    const uint32_t off = sw[warp];
    for (int i = a0 + lane; i < a1; i += 32) a[i] += off;
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Block-wide stable LSD radix sort of n <= CAP (key, value) pairs held in
// shared memory.  Each warp owns a contiguous chunk and walks it 32 elements
// at a time in order, so equal digits keep their order (stability):
//   pass A: warp-private digit counts and each element's rank among the
//           equal digits before it in its warp's chunk (__match_any_sync);
//   scan  : digit-major, warp-minor exclusive scan of the counts;
//   pass B: scatter to scan offset + rank.
// Digits are RB bits wide; `bits` is the key width to sort.
template <int THREADS, int CAP, int RB, typename V, bool HAS_V>
struct BlockRadix {
    static constexpr int W = THREADS / 32;
    static constexpr int BINS = 1 << RB;
    static constexpr int SCAN_EPT = BINS * W / THREADS;   // entries per thread in the count scan
    static_assert(SCAN_EPT * THREADS == BINS * W, "bins x warps must tile the block");

    struct Smem {
        uint32_t key[2][CAP];
        V val[HAS_V ? 2 : 1][HAS_V ? CAP : 1];
        uint16_t rank[CAP];
        uint32_t cnt[W * BINS];       // warp-major: cnt[w * BINS + d] (conflict-free per warp)
        uint32_t sw[33];
    };

    // Exclusive scan of the per-warp counts in digit-major, warp-minor order
    // (entry e = d * W + w lives at cnt[w * BINS + d]).
    __device__ static void scan_digit_major(Smem& s) {
        const int base = threadIdx.x * SCAN_EPT;
        uint32_t loc[SCAN_EPT];
        uint32_t sum = 0;
#pragma unroll
        for (int i = 0; i < SCAN_EPT; ++i) {
            const int e = base + i;
            loc[i] = s.cnt[(e % W) * BINS + e / W];
            sum += loc[i];
        }
        uint32_t tot;
        uint32_t pre = block_exclusive_scan<uint32_t, THREADS>(sum, s.sw, &tot);
#pragma unroll
        for (int i = 0; i < SCAN_EPT; ++i) {
            const int e = base + i;
            s.cnt[(e % W) * BINS + e / W] = pre;
            pre += loc[i];
        }
        __syncthreads();
    }

    // Sorts s.key[0][0..n) (and s.val[0]) by their low `bits` bits.
    // Returns the buffer index (0 or 1) that holds the result.
    __device__ static int sort(Smem& s, int n, int bits) {
        const int warp = threadIdx.x >> 5;
        const int lane = lane_id();
        const int chunk = ((n + W - 1) / W + 31) & ~31;
        const int lo = warp * chunk;
        const int hi = min(n, lo + chunk);
        int cur = 0;
        for (int shift = 0; shift < bits; shift += RB) {
            const uint32_t dmask = (bits - shift >= RB) ? (BINS - 1) : ((1u << (bits - shift)) - 1);
            for (int i = threadIdx.x; i < W * BINS; i += THREADS) s.cnt[i] = 0;
            __syncthreads();
            // pass A
            for (int base = lo; base < lo + chunk; base += 32) {
                const int i = base + lane;
                const bool ok = i < hi;
                const uint32_t d = ok ? ((s.key[cur][i] >> shift) & dmask) : 0xFFFFFFFFu;
                const uint32_t peers = __match_any_sync(0xffffffffu, d);
                if (ok) {
                    const uint32_t before = s.cnt[warp * BINS + d];
                    s.rank[i] = (uint16_t)(before + __popc(peers & lanemask_lt()));
                }
                __syncwarp();
                if (ok && (peers & lanemask_lt()) == 0) s.cnt[warp * BINS + d] += __popc(peers);
                __syncwarp();
            }
            __syncthreads();
            scan_digit_major(s);
            // pass B
            for (int i = lo + lane; i < hi; i += 32) {
                const uint32_t k = s.key[cur][i];
                const uint32_t d = (k >> shift) & dmask;
                const uint32_t pos = s.cnt[warp * BINS + d] + s.rank[i];
                s.key[cur ^ 1][pos] = k;
                if constexpr (HAS_V) s.val[cur ^ 1][pos] = s.val[cur][i];
            }
            __syncthreads();
            cur ^= 1;
        }
        return cur;
    }
};

// Block-wide LSD radix sort of packed elements: E = uint64_t holds
// (value << 32 | key) -- the memory image of a {key, value} record, so records
// are copied into shared memory verbatim -- and E = uint32_t a key alone.
// Elements with equal keys may come out in any order (every caller sums or
// merges them), so the first pass, over the lowest digit, need not be
// stable: it is a counting sort with block-wide counters and shared-memory
// atomics over up to U1 bits (13 with 16 warps).  The remaining bits are
// sorted by stable passes of at most 9-bit digits: each warp owns a
// contiguous chunk and walks it 32 elements at a time in order; lanes with
// equal digits are found by __match_any_sync or by ballots, counted in the
// warp's own counter row (rows padded by one word so the digit-major scan is
// free of bank conflicts).  A 26-bit key takes one 13-bit counting pass and
// two stable passes of 7 and 6 bits.
template <int THREADS, int CAP, typename E>
struct PackedRadix {
    static constexpr int W = THREADS / 32;
    static constexpr int MAXB = 9, MAXBINS = 1 << MAXB, ROW = MAXBINS + 1;
    static constexpr int MAX_EPT = (MAXBINS * W + THREADS - 1) / THREADS;
    static constexpr int RPT = (CAP + THREADS - 1) / THREADS;   // 32-element rows per warp at most
    static constexpr int CNT_WORDS = W * ROW;
    // widest first-pass digit whose block-wide counters fit the counter rows
    static constexpr int U1 = CNT_WORDS >= 8192 ? 13 : (CNT_WORDS >= 4096 ? 12 : (CNT_WORDS >= 2048 ? 11 : 10));

    struct Smem {
        E el[2][CAP];
        uint32_t cnt[CNT_WORDS];
        uint32_t sw[33];
    };

    __device__ static __forceinline__ uint32_t key_of(E e) { return (uint32_t)e; }
    __device__ static __forceinline__ uint32_t val_of(E e) {
        if constexpr (sizeof(E) == 8) return (uint32_t)(e >> 32);
        else return 1u;
    }

    // lanes of the warp whose digit equals this lane's (ok lanes only):
    // one ballot per digit bit, plus one for the ok flag
    __device__ static __forceinline__ uint32_t peers_ballot(uint32_t d, bool ok, int rb) {
        uint32_t m = __ballot_sync(0xffffffffu, ok);
        m = ok ? m : ~m;
        for (int b = 0; b < rb; ++b) {
            const bool bit = (d >> b) & 1u;
            const uint32_t v = __ballot_sync(0xffffffffu, bit);
            m &= bit ? v : ~v;
        }
        return m;
    }

    // First pass: counting sort of el[0][0..n) by the low b1 bits into
    // el[1] (block-wide counters, atomics; the order of equal digits is free).
    __device__ static void counting_pass(Smem& s, int n, int b1, DevStatus* st) {
        const int nb = 1 << b1;
        const uint32_t m1 = (uint32_t)nb - 1u;
        uint32_t* c = s.cnt;
        for (int i = threadIdx.x; i < nb; i += THREADS) c[i] = 0;
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += THREADS) atomicAdd(&c[key_of(s.el[0][i]) & m1], 1u);
        __syncthreads();
        block_scan_rows<THREADS>(c, nb, s.sw);
        for (int i = threadIdx.x; i < n; i += THREADS) {
            const E e = s.el[0][i];
            const uint32_t p = atomicAdd(&c[key_of(e) & m1], 1u);
            if (in_bounds(st, p, (uint64_t)n, 107)) s.el[1][p] = e;      // site 107: counting-pass position
        }
        __syncthreads();
    }

    // Ranking within a 32-element row of a stable pass: lanes with equal
    // digits are found with __match_any_sync (executed on the ADU), or with
    // one ballot per digit bit (ALU).  match: 0 = by digit width (alternating
    // for 9-bit digits, __match_any_sync for narrower ones), 1 =
    // __match_any_sync, 2 = ballots, 3 = the two alternately by row, so that
    // the ADU and ALU pipes share the work.
    // Sorts s.el[0][0..n) by the low `bits` bits of the key; returns the
    // buffer index (0 or 1) that holds the result.
    __device__ static int sort(Smem& s, int n, int bits, int match = 0, DevStatus* st = nullptr) {
        if (bits <= 0 || n <= 1) return 0;
        const int warp = threadIdx.x >> 5;
        const int lane = lane_id();
        // first pass: wide enough for the leaf's size, at most U1 bits
        const int b1 = min(bits, min(U1, max(8, (int)ceil_log2_u64((uint64_t)n) + 1)));
        counting_pass(s, n, b1, st);
        int cur = 1;
        const int rem = bits - b1;
        if (rem <= 0) return cur;
        const int passes = (rem + MAXB - 1) / MAXB;
        const int rb = (rem + passes - 1) / passes;
        const int bins = 1 << rb;
        const int total = bins * W;
        const int ept = (total + THREADS - 1) / THREADS;
        const int chunk = ((n + W - 1) / W + 31) & ~31;
        const int lo = warp * chunk;
        const int hi = min(n, lo + chunk);
        const bool ballots = match == 2;
        const bool alternate = match == 3 || (match == 0 && rb >= MAXB);
        for (int shift = b1; shift < bits; shift += rb) {
            const uint32_t dmask = (1u << min(rb, bits - shift)) - 1;
            for (int i = threadIdx.x; i < total; i += THREADS) s.cnt[(i >> rb) * ROW + (i & (bins - 1))] = 0;
            __syncthreads();
            uint32_t* row = s.cnt + warp * ROW;
            // pass A: each element's rank among the equal digits before it in
            // the warp's chunk; elements stay in registers until pass B
            E x[RPT];
            uint32_t rk[RPT];
#pragma unroll
            for (int r = 0; r < RPT; ++r) {
                const int base = lo + r * 32;
                if (base < hi) {                           // warp-uniform
                    const int i = base + lane;
                    const bool ok = i < hi;
                    x[r] = ok ? s.el[cur][i] : E(0);
                    const uint32_t d = (key_of(x[r]) >> shift) & dmask;
                    const bool bal = alternate ? (r & 1) != 0 : ballots;
                    const uint32_t peers = bal ? peers_ballot(d, ok, rb)
                                               : __match_any_sync(0xffffffffu, ok ? d : 0xFFFFFFFFu);
                    const uint32_t below = __popc(peers & lanemask_lt());
                    // the warp is converged here (no branch since the last
                    // __syncwarp), so every lane reads before its group's leader writes
                    const uint32_t before = row[ok ? d : 0];
                    rk[r] = before + below;
                    if (ok && below == 0) row[d] = before + __popc(peers);
                    __syncwarp();
                }
            }
            __syncthreads();
            {
                // exclusive scan in digit-major, warp-minor order
                const int b0 = threadIdx.x * ept;
                uint32_t loc[MAX_EPT];
                uint32_t sum = 0;
#pragma unroll
                for (int k = 0; k < MAX_EPT; ++k) {
                    loc[k] = 0;
                    const int e = b0 + k;
                    if (k < ept && e < total) {
                        loc[k] = s.cnt[(e % W) * ROW + e / W];
                        sum += loc[k];
                    }
                }
                uint32_t tot;
                uint32_t pre = block_exclusive_scan<uint32_t, THREADS>(sum, s.sw, &tot);
#pragma unroll
                for (int k = 0; k < MAX_EPT; ++k) {
                    const int e = b0 + k;
                    if (k < ept && e < total) {
                        s.cnt[(e % W) * ROW + e / W] = pre;
                        pre += loc[k];
                    }
                }
                __syncthreads();
            }
            // pass B: scatter to digit offset + rank
#pragma unroll
            for (int r = 0; r < RPT; ++r) {
                const int i = lo + r * 32 + lane;
                if (i < hi) {
                    const uint32_t d = (key_of(x[r]) >> shift) & dmask;
                    const uint32_t p = row[d] + rk[r];
                    if (in_bounds(st, p, (uint64_t)n, 108)) s.el[cur ^ 1][p] = x[r];   // site 108: stable-pass position
                }
            }
            __syncthreads();
            cur ^= 1;
        }
        return cur;
    }
};

}  // namespace hpa
