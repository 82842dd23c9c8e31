/* hpa.h -- GPU PC-sample analysis on one GB300 (sm_103a).
 *
 * C ABI of libhpa.so.  The library attributes GPU PC samples to the program
 * structure of a GPU binary, aggregates them into exact raw metrics per
 * (launch context, structure node, stall reason), splits GPU function costs
 * among call sites to form approximate GPU calling context trees, propagates
 * inclusive metrics, and derives cross-profile statistics.  The operations
 * follow "Measurement and Analysis of GPU-accelerated Applications with
 * HPCToolkit" (Zhou et al., arXiv 2109.06931); each entry point cites the
 * section that defines it.
 *
 * Conventions
 *  - Every call returns an hpa_status.  No call aborts, traps or throws.
 *  - Device work is enqueued on the handle's CUDA stream and runs
 *    asynchronously.  Errors found on the host return at once; errors found
 *    by a kernel (an invalid sample, a full output, a timed-out wait) are
 *    recorded in a device status word and returned by hpa_sync().
 *  - "device" arrays live in the handle's GPU memory and are owned by the
 *    caller; they must stay valid until hpa_sync() returns.  "host" arrays
 *    are read or written before the call returns.
 *  - Identifiers: launch-context ids are uint32 in [0, n_ctx); structure node
 *    ids are uint32 in [0, n_nodes); function ids in [0, n_funcs).
 *  - One handle per host thread.
 */
#ifndef HPA_H
#define HPA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t hpa_status;
#define HPA_OK                0
#define HPA_E_INVALID_ARG     1  /* bad pointer, size or option                    */
#define HPA_E_INVALID_TABLE   2  /* structure / call graph / CCT fails validation   */
#define HPA_E_INVALID_SAMPLE  3  /* a record has ctx >= n_ctx or stall >= n_stall   */
#define HPA_E_CAPACITY        4  /* an output array is too small; *needed is set   */
#define HPA_E_OOM             5  /* device memory could not be reserved             */
#define HPA_E_CUDA            6  /* a CUDA runtime call failed                      */
#define HPA_E_TIMEOUT         7  /* a bounded device wait gave up                   */
#define HPA_E_INTERNAL        8  /* internal invariant violated (a bug)             */
#define HPA_PENDING           9  /* a served request has not completed yet           */

#define HPA_UNKNOWN_NODE 0xFFFFFFFFu  /* node of a PC covered by no range          */
#define HPA_NO_PARENT    0xFFFFFFFFu  /* parent of a root                          */
#define HPA_MAX_STALL    32u          /* stall reasons per sample: [0, 32)         */

/* structure node kinds (Section 5: functions, inlined code, loops, lines) */
enum { HPA_NODE_FUNC = 0, HPA_NODE_INLINE = 1, HPA_NODE_LOOP = 2, HPA_NODE_LINE = 3, HPA_NODE_CALL = 4 };

/* call-edge flags of the GPU calling context tree (Section 6.3) */
enum { HPA_EDGE_FIXUP = 1,      /* weight 1 assigned by the step-2 zero-weight rule          */
       HPA_EDGE_FIXUP2 = 2,     /* weight 1 assigned by the same rule on the SCC-collapsed graph */
       HPA_EDGE_INTRA_SCC = 4   /* edge inside one recursive SCC: removed, share 0          */ };

typedef struct hpa_handle hpa_handle;

/* Options of a handle.  Zero-initialised fields take their defaults. */
typedef struct {
    uint32_t issued_mask;   /* stall reasons that count as "issued" (not stalled) in the warp
                               issue rate W; default 0x1 (reason 0)                        */
    uint32_t leaf_capacity; /* records per shared-memory leaf of the aggregation (4096 or
                               10240); 0 = chosen per call from samples per context, or by
                               hpa_tune                                                     */
    uint32_t timeout_iters; /* iteration limit of every bounded device wait; 0 = 1<<22     */
    uint32_t cursor_pad;    /* spacing of the per-context scatter cursors: 0 = 8 words for
                               up to 65,536 groups, else 1; n > 0 = 2^(n-1) words          */
    uint32_t leaf_ranking;  /* equal-digit search of the leaf radix sort: 0 = by digit width
                               (3 for 9-bit digits, else 1), 1 = __match_any_sync,
                               2 = ballots, 3 = the two alternately, row by row             */
    uint32_t grouping;      /* grouping of records by context: 0 = automatic (per-part
                               counters when every buffer has <= 4096 contexts, else
                               per-context cursors), 1 = per-context cursors always         */
    uint32_t small_leaves;  /* leaves of <= 1024 records in a separate kernel of 128-thread
                               CTAs: 0 = automatic (when a call averages fewer than 64
                               samples per context), 1 = never, 2 = always                  */
    uint32_t leaf_hash;     /* aggregation inside a leaf: 0 = radix sort of the records,
                               1 = shared-memory hash table first, then a sort of the
                               distinct keys (falls back to the sort for a leaf with too
                               many distinct keys); pays off when samples repeat keys     */
    uint32_t leaf_emit;     /* placement of the output keys: 0 = a separate pass after the
                               leaves, 1 = a leaf writes its keys itself when the keys of
                               the leaves before it are already counted (the others are
                               left to the separate pass)                                */
} hpa_options;

/* Program structure of one GPU binary (Section 5).  HOST arrays, copied into
 * library-owned device memory by hpa_load_structure.
 *  - ranges: half-open [range_lo[i], range_hi[i]) of relocated, binary-wide
 *    unique instruction addresses (Section 5: each GPU function is relocated
 *    to a unique address), sorted by lo, non-empty and pairwise disjoint
 *    (overlapping functions are split into disjoint ranges, Section 5).
 *    range_hi[n-1] - range_lo[0] must be < 2^32.  range_node[i] is the
 *    structure node (usually a LINE or CALL node) that owns the range.
 *  - nodes: a forest; node_parent[v] is HPA_NO_PARENT exactly for FUNC nodes,
 *    otherwise a node of the same function; node_func[v] is v's function.
 *    (n_nodes + 1) * n_stall must be <= 2^32.
 *  - call sites (Section 6.3 step 1): one per call instruction; cs_node[e] is
 *    the CALL node whose range is that instruction, cs_caller[e] its function,
 *    cs_callee[e] the called function.                                         */
typedef struct {
    uint64_t n_ranges;
    const uint64_t* range_lo;
    const uint64_t* range_hi;
    const uint32_t* range_node;
    uint32_t n_nodes;
    const uint32_t* node_parent;
    const uint8_t* node_kind;
    const uint32_t* node_func;
    uint32_t n_funcs;
    uint32_t n_calls;
    const uint32_t* cs_caller;
    const uint32_t* cs_callee;
    const uint32_t* cs_node;
} hpa_structure;

/* Static facts of a loaded binary. */
typedef struct {
    uint32_t n_nodes, n_funcs, n_calls;
    uint32_t n_cnodes;       /* condensed call-graph nodes V = n_funcs + non-trivial SCCs       */
    uint32_t n_scc;          /* non-trivial SCCs (>= 2 functions or a self-call)                */
    uint32_t cdag_levels;    /* levels of the condensed DAG                                      */
    uint64_t n_ranges;
    uint32_t max_depth;      /* depth of the deepest structure node (FUNC nodes have depth 0); a
                                key expands into at most max_depth + 1 inclusive records          */
    uint32_t reserved;
} hpa_binary_info;

/* One buffer of PC samples (Section 4.2: instruction address, stall reason,
 * count; plus the launch calling context the kernel ran in).  DEVICE arrays
 * (HOST arrays for the *_host entry points).  count may be NULL: every record
 * then counts 1.  Valid ids: ctx < n_ctx, stall < n_stall <= HPA_MAX_STALL.   */
typedef struct {
    uint64_t n;
    const uint64_t* pc;
    const uint32_t* ctx;
    const uint8_t* stall;
    const uint32_t* count;
    uint32_t n_ctx;
    uint32_t n_stall;
} hpa_samples;

/* Raw-metric profile: unique keys ascending by (ctx, node, stall) with their
 * exact sums.  Caller-allocated DEVICE arrays of `capacity` entries (K <= n
 * always holds, so capacity = n is always enough).  n_keys is a device uint64:
 * the number of keys written, or -- with status HPA_E_CAPACITY from hpa_sync --
 * the number needed.  total / unknown (device uint64[n_stall], may be NULL)
 * receive the per-stall sum of all counts and of the UNKNOWN ones.
 * n_ctx / n_stall / n_nodes are filled in by the producing call.              */
typedef struct {
    uint64_t capacity;
    uint32_t* key_ctx;
    uint32_t* key_node;
    uint8_t* key_stall;
    uint64_t* val;
    uint64_t* n_keys;
    uint64_t* total;
    uint64_t* unknown;
    uint32_t n_ctx;
    uint32_t n_stall;
    uint32_t n_nodes;     /* nodes of the binary the keys refer to */
    uint32_t reserved;
} hpa_profile;

/* Approximate GPU calling context trees of requested launch contexts
 * (Section 6.3), dense per context.  DEVICE arrays:
 *   req_ctx[n_req]                     contexts to reconstruct
 *   incl[n_req][n_cnodes][n_stall + 1] inclusive cost of each condensed node
 *                                      (last column: total over stall reasons);
 *                                      a function inside a non-trivial SCC has
 *                                      a zero row, its SCC row is n_funcs + k
 *   a[n_req][n_calls][n_stall + 1]     share of the callee's inclusive cost
 *                                      apportioned to each call site
 *   flags[n_req][n_calls]              HPA_EDGE_* bits                         */
typedef struct {
    uint32_t n_req;
    const uint32_t* req_ctx;
    float* incl;
    float* a;
    uint8_t* flags;
} hpa_gpucct;

/* GPU calling context trees of EVERY launch context of a profile (Section
 * 6.3, steps 1-4) as sparse rows: in each context only the condensed nodes
 * with a nonzero inclusive cost and the call sites with a nonzero share --
 * the part of the call graph above the context's sampled functions.  DEVICE
 * arrays, rows of context c at [node_off[c], node_off[c+1]) and
 * [edge_off[c], edge_off[c+1]), contexts in order:
 *   node_off[n_ctx + 1], edge_off[n_ctx + 1]  (may be NULL)
 *   node_id[cap_nodes]              condensed node, ascending within a context
 *   incl[cap_nodes][n_stall + 1]    its inclusive cost (last column: total)
 *   edge_id[cap_edges]              call site, ascending within a context
 *   ratio[cap_edges]                r(e) = w(e) / W(callee's condensed node);
 *                                   the share is a(e) = r(e) * incl(that node)
 *   a[cap_edges][n_stall + 1]       that share, or NULL: not written
 *   flags[cap_edges]                HPA_EDGE_FIXUP / HPA_EDGE_FIXUP2 bits
 *   counts[2]                       device uint64: rows written (nodes, call
 *                                   sites), or -- with HPA_E_CAPACITY from
 *                                   hpa_sync -- the rows needed
 * Entries without a row are exactly zero; a call site without a row has no
 * flags, apart from HPA_EDGE_INTRA_SCC (and HPA_EDGE_FIXUP) on the call sites
 * inside a recursive SCC, which never get rows.  Capacities both 0 ask for
 * the row counts only (no error; the costs are not computed then).          */
typedef struct {
    uint64_t cap_nodes;
    uint64_t cap_edges;
    uint64_t* node_off;
    uint32_t* node_id;
    float* incl;
    uint64_t* edge_off;
    uint32_t* edge_id;
    float* ratio;
    float* a;
    uint8_t* flags;
    uint64_t* counts;
} hpa_gpucct_all;

/* One context's GPU calling context tree materialised as a tree (Section
 * 6.3, step 4: apportioning the condensed call graph equals splitting it
 * into a tree whose call paths carry the product of the call-site ratios).
 * DEVICE arrays of `budget` entries, filled breadth-first: roots are the
 * condensed nodes without external callers (node order); the children of a
 * tree node for condensed node v at scale s are, for each external call site
 * e of v in call-site order, callee node h at scale s * r(e) with
 * r(e) = a(e) / incl(h) (total column), omitted when that scale or incl(h)
 * is zero.  incl[t][n_stall + 1] = incl(h) * scale.  parent / edge of a root
 * are HPA_NO_PARENT.  *n_nodes: nodes written; *truncated: 1 when the budget
 * cut the tree (the last level is cut in order).                            */
typedef struct {
    uint32_t budget;
    uint32_t* parent;
    uint32_t* cnode;
    uint32_t* edge;
    float* scale;
    float* incl;
    uint64_t* n_nodes;
    uint32_t* truncated;
} hpa_cct_tree;

/* Host calling context tree: DEVICE parent array (parent[v] < n_nodes or
 * HPA_NO_PARENT).  Launch context c is CCT node c (n_ctx <= n_nodes).        */
typedef struct {
    uint32_t n_nodes;
    const uint32_t* parent;
} hpa_cct;

/* Cross-profile derived metrics (Section 4.5) and warp issue rate
 * (Section 7).  DEVICE arrays.  Per key of the union of the profiles
 * (ascending (ctx, node, stall), `capacity` entries, count in *n_keys): sum,
 * min, max (absent = 0) and mean, population std, coefficient of variation.
 * Per context over the summed profiles: S, S_issued, W = S_issued / S and
 * frac[ctx][stall] = share of S per stall reason (NaN where S = 0).          */
typedef struct {
    uint64_t capacity;
    uint32_t* key_ctx;
    uint32_t* key_node;
    uint8_t* key_stall;
    uint64_t* sum;
    uint64_t* min;
    uint64_t* max;
    float* mean;
    float* std;
    float* cov;
    uint64_t* n_keys;
    uint32_t n_ctx;          /* contexts of the per-context arrays below */
    uint64_t* S;             /* [n_ctx] */
    uint64_t* S_issued;      /* [n_ctx] */
    float* W;                /* [n_ctx] */
    float* frac;             /* [n_ctx][n_stall] */
} hpa_derived;

/* Warp issue rate and stall shares per (launch context, function) (Section
 * 7: W = (S - S_stall) / S, read per kernel and per function).  DEVICE
 * arrays of `capacity` rows, ascending by (ctx, func), one row per pair
 * with samples (UNKNOWN samples belong to no function and are left out):
 * S = samples of the function in the context, S_issued = those whose stall
 * reason is in the handle's issued_mask, W = S_issued / S, frac[row][r] =
 * share of S in stall reason r (may be NULL).  *n_rows (device uint64): rows
 * written, or -- with HPA_E_CAPACITY from hpa_sync -- the rows needed.       */
typedef struct {
    uint64_t capacity;
    uint32_t* ctx;
    uint32_t* func;
    uint64_t* S;
    uint64_t* S_issued;
    float* W;
    float* frac;          /* [capacity][n_stall] */
    uint64_t* n_rows;
} hpa_issue_rows;

/* Ratio of two raw metrics per key (Section 4.5: a quantity known once per
 * kernel invocation, such as its registers, is recovered by dividing two raw
 * metrics that were summed over threads and ranks like any other: the
 * quantity summed over invocations, and the count of invocations).  DEVICE
 * arrays of `capacity` rows, ascending by (ctx, node, stall), one row per key
 * of the union of the numerator and the denominator profiles: num = the sum
 * of the numerator profiles' values of the key, den = the same over the
 * denominator profiles (0 where absent), ratio = num / den computed in FP64
 * and rounded once to FP32, NaN where den = 0.  *n_keys (device uint64): rows
 * written, or -- with HPA_E_CAPACITY from hpa_sync -- the rows needed.       */
typedef struct {
    uint64_t capacity;
    uint32_t* key_ctx;
    uint32_t* key_node;
    uint8_t* key_stall;
    uint64_t* num;
    uint64_t* den;
    float* ratio;
    uint64_t* n_keys;
} hpa_ratio_rows;

/* ---- handle ------------------------------------------------------------- */

/* Create a handle on CUDA device `device` that enqueues on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  opt may be NULL.      */
hpa_status hpa_create(hpa_handle** h, int device, void* cuda_stream, const hpa_options* opt);
/* Free every library-owned device allocation of the handle. */
hpa_status hpa_destroy(hpa_handle* h);
/* Message of the last failed call on this handle ("" if none).  The string
 * stays valid until the next call on the handle.                            */
const char* hpa_last_error(hpa_handle* h);
/* Wait for the handle's stream, then return and clear the first status a
 * kernel recorded.  *bad (may be NULL) receives the number of invalid sample
 * records when the status is HPA_E_INVALID_SAMPLE.                            */
hpa_status hpa_sync(hpa_handle* h, uint64_t* bad);
/* Reserve scratch for calls of up to max_samples records and max_groups
 * contexts (summed over a batch), so that later calls allocate nothing (as
 * stream capture requires).  Calls grow the scratch themselves otherwise.     */
hpa_status hpa_reserve(hpa_handle* h, uint64_t max_samples, uint64_t max_groups);
/* Bounded device wait (failure detection): enqueue on the handle's stream a
 * kernel that polls the DEVICE word *flag until it equals `value`, at most
 * opt.timeout_iters times with about a microsecond of sleep between polls.
 * If the word never takes the value, the kernel records HPA_E_TIMEOUT
 * (reported by hpa_sync) and returns, so the stream moves on and the context
 * stays usable.  Use: the handle's work on a buffer waits for the ready flag
 * of whatever produced it -- set by work ordered before the wait, or by the
 * host in mapped memory.  It must not wait for a kernel that only runs
 * after it (nothing guarantees two kernels run at the same time).          */
hpa_status hpa_wait_flag(hpa_handle* h, const uint32_t* flag, uint32_t value);
/* Number of kernels the handle has launched so far. */
uint64_t hpa_kernel_launches(hpa_handle* h);
/* How this library was built: bit 0 (HPA_BUILD_CHECKED) set in the
 * bounds-checked flavour (compiled with -DHPA_CHECKED), in which every index
 * that a kernel computes from counters, scans or data is checked against the
 * array it indexes; a violation skips the access and makes the call fail at
 * hpa_sync with HPA_E_INTERNAL (the detail names the site).  No handle needed. */
#define HPA_BUILD_CHECKED 1u
uint32_t hpa_build_flags(void);
/* Per-phase timing of the aggregation pipeline with CUDA events recorded on
 * the handle's stream between its kernels (enable != 0 starts a fresh
 * accumulation; 0 stops).  Phases: 0 group histogram and plan, 1 attribute +
 * scatter, 2 big-group split, 3 leaf sort/reduce, 4 emit.                    */
hpa_status hpa_set_phase_timing(hpa_handle* h, int enable);
/* After hpa_sync: ms[i] = total milliseconds of phase i over `*calls` timed
 * calls (i < n_max).  Returns HPA_OK; *n_phases receives the phase count.    */
hpa_status hpa_phase_times(hpa_handle* h, uint32_t n_max, double* ms, uint64_t* calls, uint32_t* n_phases);

/* ---- structure (Section 5, Section 6.3 steps 1 and 3) ------------------- */

/* Validate and load one binary's structure; *binary_id names it afterwards.
 * Validation: ranges sorted, non-empty, disjoint, span < 2^32; parents
 * in range and of the same function, FUNC nodes exactly the roots, no cycle;
 * call sites name existing functions and CALL nodes of the caller.
 * Failure: HPA_E_INVALID_TABLE with a message.  The call also finds the
 * call graph's strongly connected components (Tarjan's algorithm) and the
 * level order of the condensed graph, which every context shares.            */
hpa_status hpa_load_structure(hpa_handle* h, const hpa_structure* s, uint32_t* binary_id);
/* The checks of hpa_load_structure alone, on the host: no handle and no GPU
 * needed.  HPA_OK, or the status hpa_load_structure would return, with its
 * reason written to msg (msg_len bytes; msg may be NULL).                   */
hpa_status hpa_validate_structure(const hpa_structure* s, char* msg, size_t msg_len);
hpa_status hpa_unload_structure(hpa_handle* h, uint32_t binary_id);
/* Facts of a loaded binary; cnode_of_func (host uint32[n_funcs], may be NULL)
 * receives each function's condensed node id.                                */
hpa_status hpa_binary_info_get(hpa_handle* h, uint32_t binary_id, hpa_binary_info* info,
                               uint32_t* cnode_of_func);

/* ---- the hot path ------------------------------------------------------- */

/* Attribute every sample to the structure node whose range holds its PC
 * (UNKNOWN if none; Sections 4.2 and 5) and sum the counts per
 * (ctx, node, stall) into the raw metrics of `out` (Section 4.5).
 * in: DEVICE arrays; out: DEVICE arrays (see hpa_profile).  An invalid record
 * makes the whole call fail at hpa_sync with HPA_E_INVALID_SAMPLE and
 * *n_keys = 0.  Counts are exact (uint64 sums).                             */
hpa_status hpa_attribute_samples(hpa_handle* h, uint32_t binary_id, const hpa_samples* in,
                                 hpa_profile* out);

/* Same as hpa_attribute_samples with HOST input and output arrays: copies the
 * samples to the device, runs, copies the keys back and synchronises.
 * out->n_keys, total and unknown are host pointers here.  Returns the final
 * status (the hpa_sync status included).                                      */
hpa_status hpa_attribute_samples_host(hpa_handle* h, uint32_t binary_id, const hpa_samples* in,
                                      hpa_profile* out);

/* hpa_attribute_samples for callers that must not allocate device memory
 * while they analyse samples.  Examples: a measurement tool that runs inside
 * the application it observes, whose device memory belongs to the
 * application's own caching allocator (an allocation by the tool would change
 * the footprint it is measuring, and may fail because the pool has taken the
 * free memory); a serving loop that shares the GPU with other work, where
 * cudaFree would synchronise the whole device.  The paper has no counterpart:
 * this is a property of the library, not of the method.  Same arguments and
 * same keys as hpa_attribute_samples; in and out are DEVICE arrays owned by
 * the caller.  The handle's leaf_capacity, leaf_ranking, leaf_hash and
 * small_leaves options apply as there; contexts are always grouped by
 * per-context cursors (grouping is ignored).  Scratch comes from one fixed
 * 48 MiB array that the library declares in device memory, present on every
 * GPU that loads the library until the process exits (about 1.5 million
 * samples with counts per call); a call that would need more returns
 * HPA_E_INVALID_ARG and enqueues nothing.  The call makes no cudaMalloc or
 * cudaFree.  Its first call on a device looks up the array's device address
 * (once per device, under a lock); make that first call before any stream
 * capture.  All calls on a device share the array and leave their contents
 * in it: calls that overlap on the GPU (different streams or handles without
 * synchronisation between them) race and corrupt each other's results.     */
hpa_status hpa_attribute_samples_noalloc(hpa_handle* h, uint32_t binary_id, const hpa_samples* in,
                                         hpa_profile* out);

/* Many sample buffers of uneven sizes, each against its own binary, in one
 * captured CUDA graph (the analogue of streaming aggregation over profiles,
 * Section 6.1).  outs[i] receives exactly what hpa_attribute_samples would
 * give for in[i] alone.  in/outs/binary_ids are HOST arrays of descriptors
 * whose data pointers are DEVICE arrays.  Status per buffer: hpa_sync reports
 * the first failure.                                                          */
hpa_status hpa_attribute_batch(hpa_handle* h, uint32_t n, const uint32_t* binary_ids,
                               const hpa_samples* in, hpa_profile* outs);

/* Autotuner of the aggregation (no counterpart in the paper: a property of
 * the library).  Runs hpa_attribute_samples on `in` under each candidate
 * configuration -- leaf_capacity 4096 / 10240, grouping 0 / 1, leaf_hash
 * 0 / 1 (sort or hash aggregation), leaf_ranking 1 / 3: HPA_TUNE_CANDIDATES
 * in all, in that nesting order -- timing each
 * with CUDA events on the handle's stream (one untimed run, then `reps`
 * timed runs, 0 = 2), and keeps the fastest in the handle's options for the
 * calls that follow.  in/out as for hpa_attribute_samples; out holds the
 * last candidate's result.  best (may be null) receives the chosen options;
 * ms (may be null, HPA_TUNE_CANDIDATES floats) the mean time of each
 * candidate.  Synchronous: returns after the last run has finished.  Every
 * candidate computes the same keys; only their speed differs.               */
#define HPA_TUNE_CANDIDATES 16
hpa_status hpa_tune(hpa_handle* h, uint32_t binary_id, const hpa_samples* in, hpa_profile* out, uint32_t reps,
                    hpa_options* best, float* ms);

/* Approximate GPU calling context tree per requested context (Section 6.3,
 * steps 1-4): call-site weights from the samples of call instructions, the
 * step-2 zero-weight fix-up, SCC collapse, and gprof-style apportioning of
 * each condensed node's inclusive cost among its call sites.  p: a profile of
 * this binary produced by hpa_attribute_samples (device keys).  FP32 results
 * from FP64 accumulation of exact integer counts.                            */
hpa_status hpa_apportion_callgraph(hpa_handle* h, uint32_t binary_id, const hpa_profile* p,
                                   hpa_gpucct* out);

/* The same reconstruction (Section 6.3, steps 1-4) for every launch context
 * 0..p->n_ctx-1 of the profile in one call, as sparse rows (hpa_gpucct_all).
 * Inclusive costs are summed in double-float arithmetic from exact integer
 * counts and rounded once to FP32 per stored value.  Errors at hpa_sync:
 * HPA_E_CAPACITY (counts holds the rows needed; rows of the contexts that
 * fit may be written), HPA_E_INVALID_ARG (a key outside the binary).        */
hpa_status hpa_apportion_all(hpa_handle* h, uint32_t binary_id, const hpa_profile* p, hpa_gpucct_all* out);

/* Warp issue rate and stall shares per (launch context, function) of a
 * profile of this binary (Section 7; see hpa_issue_rows).  The keys are
 * regrouped by (context, function, stall) with exact 64-bit sums; each row's
 * W and shares are rounded once to FP32.  A key outside the binary (node or
 * stall) fails the call at hpa_sync with HPA_E_INVALID_SAMPLE.               */
hpa_status hpa_issue_by_function(hpa_handle* h, uint32_t binary_id, const hpa_profile* p, hpa_issue_rows* out);

/* Ratio of two raw metrics (Section 4.5; see hpa_ratio_rows) over profiles of
 * this binary: num[0..n_num) are the numerator group, den[0..n_den) the
 * denominator group (HOST arrays of profile descriptors with DEVICE data;
 * either group may be empty, not both).  Sums are exact (64-bit).  A key
 * outside the binary or the profiles' n_ctx / n_stall fails the call at
 * hpa_sync with HPA_E_INVALID_SAMPLE.                                         */
hpa_status hpa_ratio_of_sums(hpa_handle* h, uint32_t binary_id, const hpa_profile* const* num, uint32_t n_num,
                             const hpa_profile* const* den, uint32_t n_den, hpa_ratio_rows* out);

/* Inclusive metrics (Section 6.1, statistic generation).
 *  tree_out (may be NULL): for every key of p, its value is added to its node
 *    and every structure ancestor up to the function node; output keys
 *    ascending by (ctx, node, stall) with exact sums, capacity rules of
 *    hpa_profile (capacity = p's key count * (tree depth + 1) is enough).
 *  cct, cct_out (may be NULL): cct_out[v][stall] (DEVICE uint64[n_nodes][n_stall])
 *    = sum of p's values whose context lies in CCT node v's subtree.        */
hpa_status hpa_propagate_inclusive(hpa_handle* h, uint32_t binary_id, const hpa_profile* p,
                                   hpa_profile* tree_out, const hpa_cct* cct, uint64_t* cct_out);

/* Materialise the GPU calling context tree of requested context q of an
 * apportioning result g (hpa_apportion_callgraph of this binary with
 * n_stall stall reasons); see hpa_cct_tree.  Scales accumulate in FP64.    */
hpa_status hpa_expand_gpucct(hpa_handle* h, uint32_t binary_id, const hpa_gpucct* g, uint32_t n_stall,
                             uint32_t q, hpa_cct_tree* out);

/* Flat view of a profile (Section 7: costs shown by static program structure
 * alone, regardless of calling context): out keys (ctx = 0, node, stall, val)
 * with val = the sum over every context of p's values for that (node, stall),
 * ascending by (node, stall), UNKNOWN last; totals / unknown summed likewise.
 * p: a profile of this binary (device keys); out: device arrays as for
 * hpa_attribute_samples, n_ctx = 1.  Apportioning this profile with context
 * 0 requested gives the GPU calling context tree of all contexts pooled.
 * Needs (n_nodes + 1) * 2^stall_bits <= 2^28 (a dense accumulator of that
 * many uint64 in the handle's scratch); HPA_E_CAPACITY (at hpa_sync) when
 * out->capacity is too small, with *out->n_keys the size needed.            */
hpa_status hpa_flat_profile(hpa_handle* h, uint32_t binary_id, const hpa_profile* p, hpa_profile* out);

/* Sparse layouts of several profiles (Section 6.2), built on the device.  A
 * calling context is a (launch context, structure node) pair, a metric a
 * stall reason, a profile one input key list (device keys of one binary, as
 * produced by hpa_attribute_samples).  Outputs are caller-allocated DEVICE
 * arrays with capacities; counts (DEVICE) receives the sizes needed, and
 * HPA_E_CAPACITY (at hpa_sync) reports an array too small.
 *
 * CMS, context-major: planes = contexts of the union of the profiles in
 * (ctx, node) order; plane_off[i] .. plane_off[i + 1] index the plane's
 * non-empty metrics (metric_id, ascending), the sparse metric index;
 * metric_off[k] .. metric_off[k + 1] index its (pid, val) entries, one per
 * profile holding that (context, metric), ascending by profile.
 * counts[0..2] = planes, metric entries, values.  Needs
 * (n_nodes + 1) * 2^stall_bits * 2^ceil(log2 n_profiles) <= 2^32.          */
typedef struct {
    uint64_t cap_planes, cap_metrics, cap_values;
    uint32_t* plane_ctx;
    uint32_t* plane_node;
    uint64_t* plane_off;      /* [cap_planes + 1]  */
    uint8_t* metric_id;
    uint64_t* metric_off;     /* [cap_metrics + 1] */
    uint32_t* pid;
    uint64_t* val;
    uint64_t* counts;         /* [3] */
} hpa_cms;
hpa_status hpa_build_cms(hpa_handle* h, const hpa_profile* const* ps, uint32_t n_profiles, hpa_cms* out);

/* PMS, profile-major: prof_off[p] .. prof_off[p + 1] index profile p's
 * planes (its contexts in (ctx, node) order); plane_off[i] .. plane_off[i +
 * 1] index the plane's (metric_id, val) entries, ascending by metric.
 * counts[0..1] = planes, values.                                            */
typedef struct {
    uint64_t cap_planes, cap_values;
    uint64_t* prof_off;       /* [n_profiles + 1]  */
    uint32_t* plane_ctx;
    uint32_t* plane_node;
    uint64_t* plane_off;      /* [cap_planes + 1]  */
    uint8_t* metric_id;
    uint64_t* val;
    uint64_t* counts;         /* [2] */
} hpa_pms;
hpa_status hpa_build_pms(hpa_handle* h, const hpa_profile* const* ps, uint32_t n_profiles, hpa_pms* out);

/* Call-path profile unification (Section 6.1): the calling context trees of
 * several profiles merged into one.  Input CCT p: DEVICE arrays of n_nodes
 * entries -- parent (index in the same CCT, smaller than the node's own, or
 * HPA_NO_PARENT for a root), load module (< 0xFFFF) and offset (< 2^48) of
 * the node's call site.  A merged node is identified by its merged parent
 * and its (module, offset).  Output (DEVICE): uid[i] for every input node,
 * the CCTs concatenated in order; the merged tree's parent / module / offset
 * (capacity entries), numbered in the order of first occurrence in that
 * concatenation (so parents come before their children); *n_unified its
 * size.  Total nodes in [1, 2^31).  The call waits once on the handle's
 * stream (it reads the deepest level back to size the level loop), so it
 * cannot be captured into a graph.  Errors at hpa_sync: HPA_E_INVALID_TABLE
 * for a parent that does not precede its node or a site out of range (the
 * outputs are then unspecified), HPA_E_CAPACITY for a small capacity.       */
typedef struct {
    uint32_t n_nodes;
    const uint32_t* parent;
    const uint16_t* module;
    const uint64_t* offset;
} hpa_cct_nodes;
typedef struct {
    uint32_t capacity;
    uint32_t* uid;
    uint32_t* parent;
    uint16_t* module;
    uint64_t* offset;
    uint64_t* n_unified;
} hpa_cct_unified;
hpa_status hpa_unify_ccts(hpa_handle* h, const hpa_cct_nodes* ccts, uint32_t n, hpa_cct_unified* out);

/* Bottom-up view of a profile (Section 7): the costs of each function
 * divided among the calling contexts in which it is called.  The view's
 * roots are the functions of p's structure nodes (UNKNOWN keys belong to no
 * function).  Below a function, one node per caller chain: the call sites
 * met walking up `cct` from a key's launch context c (CCT node c: its own
 * call site first, then its parent's, up to the root's), cut after `levels`
 * sites; level k (0 = the functions) holds the chains of k sites, and a
 * node's children extend its chain by one site.  A node's value per stall
 * reason is the sum of p's values of its function over the contexts whose
 * chain begins with the node's chain (exact, 64-bit).
 * cct: DEVICE arrays as for hpa_unify_ccts (a parent precedes its node;
 * module < 0xFFFF, offset < 2^48), n_nodes >= p->n_ctx.  Output, DEVICE:
 * nodes level by level and within a level in the order of the first key of
 * p that reaches them; parent (HPA_NO_PARENT for a function), func, and the
 * call site (module, offset) of the chain's last site (0xFFFF, 0 for a
 * function); level_off[k] .. level_off[k + 1] (may be NULL; levels + 2
 * entries) are level k's nodes; values (val_node, val_stall, val) ascending
 * by (node, stall), zero values omitted.  counts[0..1] = nodes, values
 * needed; HPA_E_CAPACITY (at hpa_sync) for an array too small, after which
 * the arrays hold a prefix.  HPA_E_INVALID_TABLE (at hpa_sync) for a tree
 * that breaks the rules above.  Scratch: about 24 B per key of p's capacity
 * plus a table of 12 B per slot for a power of two >= 2 max(keys, tree
 * nodes).  No host synchronisation.                                         */
typedef struct {
    uint32_t levels;          /* call sites per chain, <= 1024 */
    uint64_t cap_nodes, cap_values;
    uint32_t* parent;         /* [cap_nodes] */
    uint32_t* func;
    uint16_t* module;
    uint64_t* offset;
    uint64_t* level_off;      /* [levels + 2] or NULL */
    uint32_t* val_node;       /* [cap_values] */
    uint8_t* val_stall;
    uint64_t* val;
    uint64_t* counts;         /* [2] */
} hpa_bottom_up;
hpa_status hpa_bottom_up_view(hpa_handle* h, uint32_t binary_id, const hpa_profile* p, const hpa_cct_nodes* cct,
                              hpa_bottom_up* out);

/* Derived metrics over n_profiles profiles (Section 4.5) and the warp issue
 * rate per context (Section 7, W = (S - S_stall) / S with the handle's
 * issued_mask).  ps: HOST array of profile descriptors with DEVICE data.    */
hpa_status hpa_derive_metrics(hpa_handle* h, const hpa_profile* const* ps, uint32_t n_profiles,
                              hpa_derived* out);

/* ---- serving ---------------------------------------------------------- */

/* A request loop over sample buffers that arrive over time (the serving
 * analogue of streaming aggregation, Section 6.1).  Requests are admitted in
 * arrival order while their device bytes fit in a reserved pool of
 * mem_cap_bytes (admission by free device memory); admitted requests form
 * batches that run as one batched aggregation while the next batch's samples
 * are copied in and the previous batch's keys are copied out.  Structure
 * tables stay resident in the handle; results are written to the host arrays
 * given at submit.  The server owns the handle while it exists: make no other
 * call on that handle until hpa_server_destroy.                               */
typedef struct hpa_server hpa_server;
typedef struct {
    uint64_t mem_cap_bytes;  /* device pool for admitted requests; 0 = 60 GiB    */
    uint32_t max_batch;      /* requests per batch; 0 = 64                      */
    uint32_t max_inflight;   /* batches between copy-in and copy-out; 0 = 3     */
    uint32_t reserved[4];
} hpa_server_options;
typedef struct {
    uint64_t submitted, completed, rejected, samples, batches;
    double p50_ms, p99_ms, max_ms, mean_ms;   /* latency: submit -> result in host arrays */
    double busy_s;                            /* first admission -> last completion        */
    /* per batch, mean milliseconds (CUDA events): samples copied in; waiting
     * for the device after they arrived; computing; keys ready but not yet
     * being copied out; copying out.  launch_ms: host time to admit a batch
     * and enqueue its work.                                                  */
    double h2d_ms, wait_compute_ms, compute_ms, wait_d2h_ms, d2h_ms, launch_ms;
} hpa_server_stats;

hpa_status hpa_server_create(hpa_handle* h, const hpa_server_options* opt, hpa_server** out);
/* Queue one request: in holds HOST sample arrays (pinned for full speed), out
 * HOST key arrays (out->n_keys a host uint64); both must stay valid until the
 * request completes.  Results equal hpa_attribute_samples on the same
 * samples.  *ticket names the request.                                       */
hpa_status hpa_server_submit(hpa_server* s, uint32_t binary_id, const hpa_samples* in, hpa_profile* out,
                             uint64_t* ticket);
/* HPA_PENDING while the request runs (waiting up to wait_ms first), else its
 * final status (HPA_OK, HPA_E_CAPACITY, HPA_E_OOM if it can never fit); a
 * completed ticket is forgotten after it has been reported once.            */
hpa_status hpa_server_poll(hpa_server* s, uint64_t ticket, int wait_ms);
hpa_status hpa_server_stats_get(hpa_server* s, hpa_server_stats* st);
/* Finish every queued request, then free the server (not the handle).      */
hpa_status hpa_server_destroy(hpa_server* s);

#ifdef __cplusplus
}
#endif
#endif /* HPA_H */
