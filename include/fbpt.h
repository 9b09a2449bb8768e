/*
 * fbpt.h -- C ABI of libfbpt: fused breadth-first probabilistic traversals
 * (BPTs) on one GB300 GPU, producing reverse-reachable (RR) sets under the
 * independent-cascade (IC) model and greedy max-coverage seed sets.
 *
 * Method: Neff et al., "Fused Breadth-First Probabilistic Traversals on
 * Distributed GPU Systems" (arXiv 2311.10201).  Section 2 defines the
 * problem (Definition 1, influence maximization; Definition 2, RR sets) and
 * the IC model; Section 3 and Listing 1 give the fused traversal, in which the
 * traversals of many samples share one frontier of per-vertex colour masks;
 * Section 9 names direction switching, hybrid queue/scan frontiers, dynamic
 * colour counts and mid-traversal refill as future work, which the scheduler
 * here implements.
 *
 * Conventions shared by every entry point
 *   - Every function returns FBPT_OK (0) or a negative FBPT_E* status; on
 *     failure fbpt_last_error() (thread-local) holds a one-line message.
 *     No C++ exception crosses this boundary.
 *   - "device" pointers are CUDA global-memory addresses on the current
 *     device; "host" pointers are ordinary (pageable or pinned) memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls enqueue work on it; functions that return host results
 *     synchronize it before returning.
 *
 * Bit-level contract (fixed; every output is a pure function of it):
 *   Graph: in-edge CSR.  row_ptr[n+1] (uint64, row_ptr[0] = 0, non-decreasing,
 *     row_ptr[n] = m), col[m] (uint32 < n): row v lists the sources w of the
 *     edges w -> v.  Edge id e = index into col.  thr[m] (uint32) =
 *     floor(p(e) * 2^32); 0xFFFFFFFF marks p(e) = 1 (always live).
 *   Philox4x32-10 (Salmon et al., SC'11), key = (lo32(seed), hi32(seed)).
 *   Liveness of edge e for sample s (Listing 1's per-colour, per-edge draw
 *     "random(0,1) > e.prob"): out = Philox(ctr = (lo32(s), hi32(s),
 *     lo32(e >> 2), hi32(e >> 2))); e is live for s iff thr[e] == 0xFFFFFFFF
 *     or out[e & 3] < thr[e].  One Philox call serves four consecutive edges
 *     of one sample.
 *   Start vertex of sample s (Section 3: starts uniform over V):
 *     out = Philox(ctr = (lo32(s), hi32(s), 0, 0x80000000)),
 *     start(s) = floor(((out[1] << 32) | out[0]) * n / 2^64).
 *   RR set of s (Definition 2): every w with a path w -> ... -> start(s)
 *     whose edges are all live for s.  Rows are in sample-id order, vertices
 *     strictly ascending; start(s) is always in its own row.
 *   Greedy (Section 2, max-k-cover over the RR sets): each pick takes the
 *     vertex contained in the most not-yet-covered RR sets, the smallest
 *     vertex id on ties; once every set is covered, the smallest unselected
 *     id.  Exactly k seeds.
 */
#ifndef FBPT_H
#define FBPT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FBPT_VERSION 1

enum fbpt_status {
    FBPT_OK = 0,
    FBPT_EINVAL = -1,       /* bad argument or malformed graph */
    FBPT_ENOMEM = -2,       /* a device or host allocation failed */
    FBPT_ECUDA = -3,        /* a CUDA runtime call failed */
    FBPT_ETIMEOUT = -4,     /* a bounded device wait gave up */
    FBPT_EUNSUPPORTED = -5, /* option combination not available */
    FBPT_EDEVICE = -6       /* a kernel's own bounds check tripped */
};

enum fbpt_mem_kind { FBPT_MEM_HOST = 0, FBPT_MEM_DEVICE = 1 };

/* Level schedule: how each level's frontier is expanded. */
enum fbpt_schedule {
    FBPT_SCHED_PUSH = 0,      /* always push over in-edges of frontier vertices */
    FBPT_SCHED_PULL = 1,      /* always pull over out-edges of unvisited vertices */
    FBPT_SCHED_HEURISTIC = 2, /* degree-ratio rule picks push or pull per level */
    FBPT_SCHED_LEARNED = 3,   /* policy network picks, heuristic as fallback */
    FBPT_SCHED_FILTERED = 4   /* always push, skipping draws for colours the source already has */
};

/* How the level loop is driven. */
enum fbpt_launch {
    FBPT_LAUNCH_HOST = 0,  /* host launches each level and reads the loop condition back, one
                              level queued ahead of the one it waits for (that level's kernels
                              return at once if the run has ended) */
    FBPT_LAUNCH_GRAPH = 1, /* per-level kernels looped inside one CUDA graph (WHILE conditional node) */
    FBPT_LAUNCH_PERSISTENT = 2 /* one cooperative persistent kernel; levels separated by bounded
                                  grid barriers (FBPT_ETIMEOUT if a wait gives up) */
};

/* How the vertices reached at a level are gathered for the commit (Section
 * 9 (a): a hybrid of a queue and a scan of the frontier). */
enum fbpt_compaction {
    FBPT_COMPACT_QUEUE = 0, /* the expand appends each newly reached vertex to a pending list (an
                               atomic with a returned value per new vertex) */
    FBPT_COMPACT_SCAN = 1   /* the expand only sets bits (no returned value, no list); the commit
                               scans every vertex's word-occupancy mask for the reached ones.
                               Pull levels always use the queue */
};

/* When a colour lane takes its next sample. */
enum fbpt_refill {
    FBPT_REFILL_LANE = 0,  /* as soon as the lane's traversal ends (mid-traversal injection) */
    FBPT_REFILL_BATCH = 1  /* only when every lane of the row has finished: the plain fused
                              algorithm with 64 * words * slots colours per group */
};

/* Diffusion model of the RR sets (Section 2 names IC and LT). */
enum fbpt_model {
    FBPT_MODEL_IC = 0,  /* independent cascade: edge e live for sample s by its own draw (contract above) */
    FBPT_MODEL_LT = 1   /* linear threshold, live-edge form: each vertex keeps at most one in-edge.
                           thr[e] is the weight w(e) = thr[e] / 2^32 (0xFFFFFFFF read as 1), and a
                           row's weights must sum to at most 1 (FBPT_EINVAL otherwise).  For sample
                           s, vertex v draws r = out[0] of Philox(ctr = (lo32(s), hi32(s), v,
                           0x40000000)) and keeps the first edge e of its row with
                           r < w(first) + ... + w(e) (in units of 2^-32), none if r is beyond the
                           row's total.  The RR set of s is the walk start(s) <- u1 <- u2 ... along
                           the kept in-edges, ending at a vertex that kept none or at one already
                           on the walk.  Levels are push only; the unfused form is not offered */
};

/* One row per level of a sampling run, filled when fbpt_opts.trace is set.
 * The schedule policy is trained on these rows (features of a level and the
 * time each phase took). */
typedef struct fbpt_trace_row {
    uint64_t level;          /* level index within the run */
    uint64_t units;          /* frontier units expanded at this level */
    uint64_t groups;         /* their 4-edge groups (expand work items) */
    uint64_t colours;        /* colour bits carried by the units */
    uint64_t pending;        /* vertices whose next row changed (commit work items) */
    uint64_t active_lanes;   /* lanes still traversing after this level */
    uint64_t finished_lanes; /* lanes whose sample ended at this level */
    uint64_t started_lanes;  /* lanes given a new sample at this level */
    uint64_t expand_ns, commit_ns, sweep_ns;  /* device time of each phase (%globaltimer) */
    uint32_t direction;      /* how this level expanded: 0 push, 1 filtered push, 2 pull */
    uint32_t frontier_lanes; /* lanes with colours in this level's frontier */
    float features[6];       /* the policy features of this level as the scheduler computed them
                                (FP64 arithmetic rounded to FP32; see the schedule policy below);
                                zero in row 0, whose level no schedule step preceded */
    float outputs[8];        /* the policy network's outputs for this level (learned schedule with a
                                policy), else zero */
    uint32_t compaction;     /* how this level gathered its reached vertices (enum fbpt_compaction) */
    uint32_t reserved;
} fbpt_trace_row;

typedef struct fbpt_graph fbpt_graph;
typedef struct fbpt_policy fbpt_policy;

typedef struct fbpt_opts {
    uint32_t words;      /* W: 64-colour mask words per batch (1, 2, 4 or 8); 0 = 8 */
    uint32_t slots;      /* batches traversed concurrently, sharing one frontier; 0 = 64 / words.
                            A vertex row holds words * slots <= 64 words, i.e. that many
                            64-colour lanes groups; each colour lane carries one sample */
    uint32_t schedule;   /* enum fbpt_schedule */
    uint32_t launch;     /* enum fbpt_launch */
    uint32_t unfused;    /* 1 = each colour expands its own copy of every edge (no fusing);
                            output is identical, only the work differs */
    uint32_t refill;     /* enum fbpt_refill */
    uint32_t blocks;     /* CTAs of each level kernel; 0 = every CTA the GPU holds at once.
                            Fewer leave room for other graphs of a batched run */
    uint32_t model;      /* enum fbpt_model (0 = IC) */
    const fbpt_policy* policy; /* used by FBPT_SCHED_LEARNED; NULL = built-in heuristic */
    void* stream;        /* cudaStream_t */
    uint64_t spin_limit; /* FBPT_LAUNCH_PERSISTENT: polls before a grid-barrier wait gives up
                            (0 = default, about a few seconds) */
    fbpt_trace_row* trace; /* host array of trace_cap rows, or NULL; levels beyond trace_cap
                              are not recorded */
    uint64_t trace_cap;
    uint32_t compaction; /* enum fbpt_compaction of the push, filtered and pull schedules; the
                            heuristic and learned schedules choose it per level */
    uint32_t reserved;   /* 0 */
} fbpt_opts;

/* RR sets as CSR in library-owned device memory (free with fbpt_rrsets_free). */
typedef struct fbpt_rrsets {
    uint64_t S;          /* rows */
    uint64_t total;      /* offsets[S] = sum of row sizes */
    uint32_t n;          /* vertices of the graph sampled */
    uint64_t* offsets;   /* device, S+1 */
    uint32_t* verts;     /* device, total; row j = verts[offsets[j] .. offsets[j+1]) ascending */
    uint32_t* starts;    /* device, S: start(first_id + j) */
    uint32_t* vcount;    /* device, n: number of rows containing v (mask popcounts) */
    void* stream;        /* stream the buffers belong to */
    void* internal;      /* library bookkeeping */
} fbpt_rrsets;

typedef struct fbpt_stats {
    uint64_t levels;              /* expand launches (ticks) */
    uint64_t batches;             /* 64*W-colour batches traversed */
    uint64_t push_levels, pull_levels;
    uint64_t units_expanded;      /* frontier vertices expanded, summed over levels */
    uint64_t edge_accesses;       /* (frontier vertex, in-edge) pairs read, summed over levels */
    uint64_t philox_calls;        /* Philox4x32-10 evaluations in expand */
    uint64_t colour_edge_visits;  /* sum over samples s and v in RR(s) of indeg(v) */
    uint64_t rr_total;            /* sum of RR set sizes */
    uint64_t overflow_reruns;     /* batches re-run after the output pool grew */
    uint64_t mask_words;          /* non-zero 64-colour mask words of expanded frontier units */
    uint64_t trace_rows;          /* rows written to fbpt_opts.trace */
    uint64_t groups_expanded;     /* 4-edge groups of the push levels' frontier units (expand work items) */
    double ms_total;              /* device time of the call on its stream (CUDA events), from
                                     the first sampling kernel to the finished CSR; workspace
                                     allocation on a graph's first use is not included */
    double ms_expand;             /* device time of the expand phase: per level, first CTA start
                                     to last CTA end (%globaltimer), summed */
    double ms_commit;             /* same for the commit phase */
    double ms_sweep;              /* same for the sweep phase (RR pairs of finished lanes) */
    double ms_expand_events;      /* FBPT_LAUNCH_HOST only: the time of each level's expand kernel
                                     (start vertices, sweep, expand) measured by CUDA events recorded
                                     around it on the run's stream, summed; the host keeps one level
                                     queued ahead, so the events bracket the kernels (0 for the other
                                     launch forms, whose levels run inside one launch) */
} fbpt_stats;

/* ---- Graphs ---------------------------------------------------------------
 * Copies the in-edge CSR and thresholds (mem_kind says where the inputs live)
 * into library-owned device memory; the caller may free its arrays on return.
 * Validates row_ptr[0] = 0, monotone rows, row_ptr[n] = m, col[e] < n
 * (FBPT_EINVAL otherwise).  n >= 1, m < 2^40.  thr is kept exactly as given. */
int fbpt_graph_create(uint32_t n, uint64_t m, const uint64_t* row_ptr, const uint32_t* col,
                      const uint32_t* thr, int mem_kind, void* stream, fbpt_graph** out);
int fbpt_graph_destroy(fbpt_graph* g);
/* n, m and device addresses of the stored arrays (any pointer may be NULL).
 * While a vertex order is set (fbpt_graph_set_order), col holds relabelled
 * sources (perm[u]); row_ptr and thr are never changed. */
int fbpt_graph_info(const fbpt_graph* g, uint32_t* n, uint64_t* m, const uint64_t** row_ptr,
                    const uint32_t** col, const uint32_t** thr);

/* ---- Vertex order (Section 5: reordering raises colour occupancy) ------------
 * The paper relabels vertices (RCM, clustering) so that vertices reached
 * together lie together, and lets the workers take start vertices from a
 * sorted list.  Here a vertex order relabels only the device state that is
 * indexed by vertex (the visited / next rows, the pending list, frontier
 * units): the in-edges keep their in-CSR positions, so every liveness draw
 * keeps its (sample id, edge index) counter and every result is unchanged.
 * RR sets, starts and counts are returned in the caller's vertex ids. */
enum fbpt_order_method {
    FBPT_ORDER_IDENTITY = 0,  /* perm[v] = v */
    FBPT_ORDER_RCM = 1,       /* reverse Cuthill-McKee over the undirected graph (u-v for every edge
                                 u -> v, u != v): per component, a breadth-first search from an
                                 unvisited vertex of least degree (ties: least id), neighbours taken
                                 by increasing (degree, id); the order is then reversed */
    FBPT_ORDER_DEGREE = 2,    /* by decreasing undirected degree, ties by id (hubs first) */
    FBPT_ORDER_RANDOM = 3,    /* a uniform permutation drawn from seed (the paper's baseline) */
    FBPT_ORDER_CLUSTER = 4    /* communities of the undirected graph contiguous (the paper's
                                 clustering order, Grappolo, is parallel Louvain): Louvain modularity
                                 optimisation (Blondel et al. 2008), vertices moved in id order to the
                                 neighbouring community of largest gain (ties: the lower community id;
                                 a vertex stays unless the gain is positive), levels aggregated until
                                 a level moves nothing (at most 8 levels; passes repeat until at
                                 most 0.1 % of the nodes move, at most 16 per level).
                                 Communities are laid out by decreasing total degree (ties: least
                                 member id), recursively by level; vertices within the finest
                                 community by decreasing degree, then id */
};
/* Host only (needs no GPU): a vertex order of the graph given by its in-edge
 * CSR (host arrays, the layout of fbpt_graph_create).  perm (n entries, caller
 * owned) receives the new label of every vertex.  FBPT_EINVAL on a null
 * array, an unknown method or a malformed CSR; FBPT_ENOMEM if the undirected
 * adjacency (2m entries) cannot be allocated. */
int fbpt_order_compute(uint32_t n, uint64_t m, const uint64_t* row_ptr, const uint32_t* col, uint32_t method,
                       uint64_t seed, uint32_t* perm);
/* Sets the vertex order of g: perm (host, n entries: perm[v] = new label of v)
 * must be a permutation of 0 .. n-1 (FBPT_EINVAL otherwise); NULL restores the
 * identity.  sorted_starts = 1 makes the samples of every later sampling call
 * take lanes in increasing order of their (relabelled) start vertex, ties by
 * sample id (Section 5's sorted start list), instead of in sample-id order.
 * Pull levels are not available while a non-identity order is set: the pull
 * schedule then fails with FBPT_EUNSUPPORTED and the heuristic and learned
 * schedules choose between push and filtered push only.  Synchronous. */
int fbpt_graph_set_order(fbpt_graph* g, const uint32_t* perm, uint32_t sorted_starts);
/* The order set on g: perm (host, n entries, may be NULL) and sorted_starts
 * (may be NULL). */
int fbpt_graph_get_order(const fbpt_graph* g, uint32_t* perm, uint32_t* sorted_starts);

/* ---- Sampling ----------------------------------------------------------------
 * RR sets of samples first_id .. first_id + S - 1 (Definition 2, computed by
 * the fused traversal of Listing 1).  Rows are in sample-id order; results
 * do not depend on opts (W, slots, schedule, launch, unfused).  out is filled
 * with library-owned device buffers.  stats may be NULL. */
int fbpt_sample(fbpt_graph* g, uint64_t seed, uint64_t first_id, uint64_t S, const fbpt_opts* opts,
                fbpt_rrsets* out, fbpt_stats* stats);

/* Many graphs in one run: graph i gets samples first_ids[i] .. + Ss[i] - 1
 * under seeds[i]; outs[i] receives its RR sets, identical to what fbpt_sample
 * gives for the same arguments.  With opts->launch FBPT_LAUNCH_HOST the graphs
 * run one after another through fbpt_sample (the plain form).  Otherwise one
 * CUDA graph holds every task as its own branch (the control block's reset, a
 * WHILE node over the level kernels, the last sweep, the control block's
 * read-back); branches of different graphs have no edges between them, so the
 * GPU runs them concurrently, and tasks that share a graph (and so its
 * workspace) are chained.  The whole batch is ONE cudaGraphLaunch.  When
 * opts->words == 0, each graph runs with the shape fbpt_autotune stored on it
 * (words, slots, refill, blocks and schedule), else the fixed default.  Tasks whose RR sets
 * outgrew their buffers run again on their own.  Traces are not recorded.  On
 * error every outs[i] is released. */
int fbpt_sample_batched(uint32_t G, fbpt_graph* const* gs, const uint64_t* seeds, const uint64_t* first_ids,
                        const uint64_t* Ss, const fbpt_opts* opts, fbpt_rrsets* outs, fbpt_stats* stats);

/* ---- Autotuner ------------------------------------------------------------------
 * Launch shape of one graph, measured by fbpt_autotune: the mask row width
 * (words * slots 64-bit words, i.e. that many 64-colour lane groups), the
 * refill mode and the CTAs per level kernel. */
typedef struct fbpt_tuning {
    uint32_t words, slots, refill, blocks;
    uint32_t candidates;      /* shapes measured */
    uint32_t schedule;        /* enum fbpt_schedule kept for this graph */
    uint64_t probe_samples;   /* samples per timed probe */
    double probe_rate;        /* samples per second of the chosen shape in its probe */
    double rr_per_sample;     /* mean RR set size seen by the probes */
} fbpt_tuning;

/* Times sampling runs of g on sample ids 0 .. P - 1 under seed, where P (in
 * [min(S, 4096), min(S, 65536)]) makes one probe take about 50 ms, measured on
 * a first run of min(S, 4096) samples.  Each shape is warmed up on P / 8
 * samples first.  Row widths 1, 2, 4, ..., 64 words (at most one lane per probe
 * sample), then the best width with 1, 1/2, 1/4 and 1/8 of the resident CTAs:
 * it keeps the fastest width, and a smaller grid only if it is more than 3%
 * faster than the best so far (a probe's few samples favour small grids more
 * than a full run does).  base supplies the schedule and policy
 * (NULL = push); when base->words is set, base->words * base->slots (slots 0
 * read as 1) caps the widths tried.  A learned (or heuristic) schedule is then
 * judged at that shape against the heuristic (or learned, with a policy): the
 * other is kept only if it is at least 3% faster; plain push (no second
 * expand kernel per level) is kept whenever it is within 3% of the best.  The result is stored on g (used by fbpt_sample_batched) and
 * copied to out (may be NULL).  Output bits never depend on the shape. */
int fbpt_autotune(fbpt_graph* g, uint64_t seed, uint64_t S, const fbpt_opts* base, fbpt_tuning* out);
/* The row width picked by the policy network instead of measured (Section 9
 * (a), dynamic colour counts): one run of sample ids 0 .. min(S, 8192) - 1 at
 * 8 words x 1 slot with lane refill and the learned schedule (base->policy,
 * required; base supplies the stream and launch form) records the network's
 * outputs 5..7 on every level, its predicted log2 ns per sample at rows of 4,
 * 16 and 64 words; *row_words receives the width whose mean over the levels
 * that had a frontier is smallest (64 if none had), scores (3 floats, may be
 * NULL) the three means.  FBPT_EINVAL for a null argument, S = 0 or no policy. */
int fbpt_policy_width(fbpt_graph* g, uint64_t seed, uint64_t S, const fbpt_opts* base, uint32_t* row_words,
                      float* scores);

/* The shape stored on g by fbpt_autotune; FBPT_EINVAL if it was never tuned. */
int fbpt_graph_tuning(const fbpt_graph* g, fbpt_tuning* out);
/* Stores a shape on g as fbpt_autotune would (words in {1, 2, 4, 8}, slots >= 1,
 * words * slots <= 64, a valid refill mode and schedule; blocks 0 = every CTA
 * the GPU holds), e.g. to run the batched form at one shape under several
 * schedules.  FBPT_EINVAL otherwise. */
int fbpt_graph_set_tuning(fbpt_graph* g, const fbpt_tuning* t);

int fbpt_rrsets_free(fbpt_rrsets* rr);
/* Host copies (any pointer may be NULL): offsets[S+1], verts[total], starts[S], vcount[n]. */
int fbpt_rrsets_copy_to_host(const fbpt_rrsets* rr, uint64_t* offsets, uint32_t* verts, uint32_t* starts,
                             uint32_t* vcount);
/* Host copy of rows first_row .. first_row + count - 1 only: offsets_host
 * receives count + 1 offsets (relative to the whole set, as in rr->offsets) and
 * verts_host their vertices, at most verts_cap of them; FBPT_EINVAL if the rows
 * are out of range or hold more than verts_cap vertices. */
int fbpt_rrsets_copy_rows(const fbpt_rrsets* rr, uint64_t first_row, uint64_t count, uint64_t* offsets_host,
                          uint32_t* verts_host, uint64_t verts_cap);

/* ---- Seed selection -------------------------------------------------------------
 * Greedy max-k-cover over rr (contract above).  seeds_host[k] receives the
 * picks in order; gains_host[k] (may be NULL) the number of RR sets each pick
 * newly covered.  k > rr->n gives FBPT_EINVAL. */
int fbpt_select_seeds(const fbpt_rrsets* rr, uint32_t k, uint32_t* seeds_host, uint64_t* gains_host);

/* The same picks and gains as fbpt_select_seeds, for callers that cannot
 * allocate device memory when they select seeds: for example a serving process
 * that gives all free device memory to its own pool at start-up, or a thread on
 * a latency-critical path that must stay clear of the allocator.  The paper has
 * no counterpart; this is a property of the library, not of the method.
 * It allocates nothing: its working memory is one fixed 64 MiB array in the
 * library's device image, which every GPU that loads libfbpt holds until the
 * process exits.  CUDA loads the library's device code lazily by default, so
 * the array is placed on a device when the first graph is created there
 * (fbpt_graph_create looks the array up for this reason); a caller that builds
 * its RR sets without a graph on that device must make one call before it
 * hands its free memory to a pool.  It needs 4*n + n + S + 20*k bytes (each
 * part rounded up to 256) and returns FBPT_EINVAL, naming the limit, beyond
 * 64 MiB.  Every call looks up the array's device address
 * (cudaGetSymbolAddress).  All calls share the array and each starts by
 * clearing it: calls whose work overlaps on the GPU (two host threads, or two
 * streams) race and give wrong seeds, so serialize them.  Work runs on
 * rr->stream; the call returns after it finishes. */
int fbpt_select_seeds_noalloc(const fbpt_rrsets* rr, uint32_t k, uint32_t* seeds_host, uint64_t* gains_host);

/* ---- Influence maximization: the IMM sampling loop -------------------------------
 * The consumer of the sampler that Section 2 describes: IMM (Tang, Shi and
 * Xiao, SIGMOD 2015) fixes the number of RR sets theta that gives a
 * (1 - 1/e - epsilon)-approximate seed set with probability at least
 * 1 - n^-ell, then runs greedy max-k-cover over them.  With natural logs,
 * ell' = ell * (1 + ln 2 / ln n), eps' = sqrt(2) * epsilon and
 * L = ln C(n, k) (the sum over i < min(k, n - k) of ln((n - i) / (i + 1))):
 *   lambda' = (2 + 2 eps'/3) (L + ell' ln n + ln log2 n) n / eps'^2,
 *   lambda* = 2 n ((1 - 1/e) alpha + beta)^2 / epsilon^2 with
 *             alpha = sqrt(ell' ln n + ln 2), beta = sqrt((1 - 1/e)(L + ell' ln n + ln 2)).
 * Rounds i = 1 .. ceil(log2 n) - 1: x = n / 2^i; the sample holds
 * theta_i = ceil(lambda' / x) RR sets (sample ids 0 .. theta_i - 1 under seed,
 * extended, never redrawn); greedy picks k seeds covering a fraction F of
 * them; if n F >= (1 + eps') x the lower bound is LB = n F / (1 + eps') and
 * the rounds stop (LB = 1 if no round succeeds).  Then theta =
 * ceil(lambda* / LB), theta RR sets are drawn afresh (sample ids right after
 * those of the estimation rounds: Chen, 2018, showed that reusing the
 * estimation sets, as the original IMM does, breaks the martingale argument
 * behind the guarantee) and the greedy seeds over them are the result.  Every sampling step is fbpt_sample
 * with opts, every selection fbpt_select_seeds.
 *
 * Needs n >= 2, 1 <= k <= n, epsilon > 0, ell > 0.  max_samples (0 = none)
 * caps the sample: FBPT_EINVAL, naming the size, if a round or theta needs
 * more.  seeds_host[k] and gains_host[k] (may be NULL) receive the final
 * picks; result (may be NULL) the sizes and bounds; stats (may be NULL)
 * accumulates over every sampling call. */
typedef struct fbpt_imm_result {
    uint64_t theta;       /* ceil(lambda* / LB) */
    uint64_t samples;     /* RR sets the final selection used (theta) */
    uint64_t first_final_id; /* sample id of the first of them (the estimation sample's size) */
    double lower_bound;   /* LB */
    double coverage;      /* fraction of those RR sets the seeds cover */
    double lambda_prime, lambda_star;
    uint32_t rounds;      /* estimation rounds run */
    uint32_t reserved;
} fbpt_imm_result;

int fbpt_imm(fbpt_graph* g, uint32_t k, double epsilon, double ell, uint64_t seed, uint64_t max_samples,
             const fbpt_opts* opts, uint32_t* seeds_host, uint64_t* gains_host, fbpt_imm_result* result,
             fbpt_stats* stats);

/* ---- Schedule policy --------------------------------------------------------------
 * A 6 -> 32 -> 32 -> 8 ReLU network (FP32) that picks, per level, how the
 * level expands and gathers its reached vertices (Section 9 (a): direction
 * switching among push, push that skips colours the source already has, and
 * pull; a queue or a scan of the frontier), and the row width of a run
 * (dynamic colour counts).  Outputs 0..4 are the predicted log2 device time of
 * the level under push, filtered push and pull with queue compaction, then
 * push and filtered push with scan compaction; the scheduler takes the
 * smallest allowed one.  Outputs 5..7 are the predicted log2 ns per sample of
 * a run at rows of 4, 16 and 64 words (fbpt_policy_width).  It changes the
 * schedule only, never a bit of the output.
 * Parameters (fbpt_policy_param_count() floats): input mean[6], input
 * scale[6] (> 0), W1[32][6], b1[32], W2[32][32], b2[32], W3[8][32], b3[8];
 * features as in fbpt_trace_row: log2(1+units), log2(1+groups),
 * log2(1+colours), log2(1+frontier_lanes), log2(1+4*groups) - log2(1+m),
 * log2(1+colours/units). */
int fbpt_policy_param_count(void);
int fbpt_policy_create(const float* params, uint64_t count, fbpt_policy** out);
int fbpt_policy_destroy(fbpt_policy* p);
int fbpt_policy_get(const fbpt_policy* p, float* params, uint64_t count);
/* Writes p's parameters to a text file, one number per line printed with
 * "%.9g" (a float32 reads back exactly): the format of the package's shipped
 * policy.  FBPT_EINVAL for a null argument or a file that cannot be written. */
int fbpt_policy_save(const fbpt_policy* p, const char* path);
/* Reads fbpt_policy_param_count() numbers separated by white space from a
 * text file into a new policy (as fbpt_policy_create).  FBPT_EINVAL if the file
 * cannot be read, holds a token that is not a number, or holds another count. */
int fbpt_policy_load(const char* path, fbpt_policy** out);

/* Training on trace rows (host arrays): features[rows][6] as above,
 * actions[rows] (the direction a level ran with), targets[rows] (its log2
 * device time in ns).  Loss: mean of (out[action] - target)^2, full-batch
 * Adam on the weights and biases for opts->steps steps (0 = 2000) at
 * opts->lr (0 = 3e-3).  init_params may be NULL: the input mean and scale
 * then come from the data and the weights from a seeded He initialisation.
 * Forward, backward and update run in the library's own CUDA kernels.
 * *out receives a new policy; *final_loss (may be NULL) its loss. */
typedef struct fbpt_train_opts {
    uint32_t steps;
    float lr;
    uint64_t seed;
    void* stream;    /* cudaStream_t the training kernels and copies run on (NULL = legacy default) */
} fbpt_train_opts;
int fbpt_policy_train(const float* features, const uint32_t* actions, const float* targets, uint64_t rows,
                      const fbpt_train_opts* opts, const float* init_params, fbpt_policy** out, float* final_loss);
/* Loss and gradient (param_count floats; zero for the input mean and scale)
 * of the parameters on the rows, computed by the training kernel on stream. */
int fbpt_policy_loss_grad(const float* params, const float* features, const uint32_t* actions,
                          const float* targets, uint64_t rows, float* loss, float* grad, void* stream);
/* One Adam update (Kingma and Ba, ICLR 2015, Algorithm 1; beta1 = 0.9,
 * beta2 = 0.999, eps = 1e-8) by the training's own kernel, at step t >= 1 with
 * learning rate lr > 0: m = beta1 m + (1 - beta1) g, v = beta2 v + (1 - beta2) g^2,
 * params -= lr (m / (1 - beta1^t)) / (sqrt(v / (1 - beta2^t)) + eps), for every
 * weight and bias; the input mean and scale (the first 12 floats) are left as
 * they are.  params, m and v (param_count floats each, host) are updated in
 * place; grad (host) is read.  Runs on stream and returns when done.
 * FBPT_EINVAL for a null array, t = 0 or lr <= 0. */
int fbpt_policy_adam_step(float* params, const float* grad, float* m, float* v, uint32_t t, float lr, void* stream);

/* ---- Building blocks exposed for verification ------------------------------------
 * Device results of the bit-level contract for given inputs (host arrays in
 * and out, count entries each): edge draws out[e & 3] for pairs (s[i], e[i]),
 * and start vertices for sample ids. */
int fbpt_edge_draws(uint64_t seed, const uint64_t* s, const uint64_t* e, uint64_t count, uint32_t* out);
int fbpt_start_vertices(uint64_t seed, const uint64_t* s, uint64_t count, uint32_t n, uint32_t* out);

/* Measured ceiling of the liveness draw (the integer-ALU roofline of the push
 * expand): a kernel that does nothing but Philox4x32-10 evaluations, round
 * keys hoisted as in the expand, calls_per_thread (>= 2) per thread over every
 * thread the GPU holds at once; three launches after one warm-up are timed
 * with CUDA events on stream.  *calls_per_s receives evaluations per second.
 * FBPT_EINVAL for a null result or calls_per_thread < 2. */
int fbpt_philox_rate(uint64_t seed, uint32_t calls_per_thread, void* stream, double* calls_per_s);

/* sizeof(fbpt_opts), sizeof(fbpt_rrsets), sizeof(fbpt_stats), sizeof(fbpt_tuning),
 * sizeof(fbpt_imm_result), sizeof(fbpt_trace_row) into sizes[0 .. min(count, 6) - 1]
 * (count >= 3), so that bindings can check their struct layouts. */
int fbpt_abi_sizes(uint64_t* sizes, int count);

const char* fbpt_last_error(void);
int fbpt_version(void);

#ifdef __cplusplus
}
#endif
#endif /* FBPT_H */
