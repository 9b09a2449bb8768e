// Internal structures of libfbpt shared by its translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace fbpt {

constexpr uint32_t kMaxWords = 64;      // 64-bit colour words per vertex row
constexpr uint32_t kMaxLanes = 64 * kMaxWords;
constexpr uint32_t kUnitBits = 26;      // list allocation counter: units in the low 26 bits
constexpr uint64_t kUnitMask = (1ull << kUnitBits) - 1;
constexpr uint32_t kSegMin = 1024;      // smallest per-lane segment (RR entries a lane keeps in its own list)
constexpr uint64_t kSegBytesMax = 2ull << 30;  // largest segment array of a workspace
// A spill-log entry packs (lane, position in the lane's row, vertex) as 12 + 26 + 26 bits.
constexpr uint32_t kSpillPosBits = 26;
constexpr uint64_t kSpillMask = (1ull << kSpillPosBits) - 1;
constexpr uint32_t kChunk = 32;         // 4-edge groups per expand chunk (one per lane)
// Frontier units with at least this many 4-edge groups are "wide": each of
// their expand chunks is 32 groups of that unit alone (the lanes share its
// colours); narrower units are packed 32 groups per chunk across units.
constexpr uint32_t kWideMin = 32;
constexpr uint32_t kWideSpan = 64;      // groups of a wide chunk: two per lane
#ifndef FBPT_COLOUR_BLOCK
#define FBPT_COLOUR_BLOCK 32
#endif
// A wide chunk draws for at most this many of its unit's colours; a unit with
// more colours has a chunk per (32 groups, block of colours), so that no chunk
// holds a warp much longer than the others.
constexpr uint32_t kColourBlock = FBPT_COLOUR_BLOCK;
constexpr uint32_t kPendBuf = 32;       // per-warp buffer of new pending vertices in the expand
#ifndef FBPT_CHUNKS_PER_GRAB
#define FBPT_CHUNKS_PER_GRAB 2
#endif
constexpr uint32_t kChunksPerGrab = FBPT_CHUNKS_PER_GRAB;  // chunks a warp takes per atomic


enum ErrorBits : uint32_t {
    kErrListOverflow = 1u,
    kErrChunkOverflow = 2u,
    kErrTickLimit = 4u,
    kErrPendOverflow = 8u,
    kErrBarrierTimeout = 16u,
    kErrSpillOverflow = 32u,
    kErrWideOverflow = 64u,   // the wide-chunk map was too small (the host grows it and reruns)
};

// How a level expands its frontier.
enum Direction : uint32_t {
    kDirPush = 0,      // push over in-edges of frontier units; draws for every frontier colour
    kDirFiltered = 1,  // push, skipping colours the source has already seen (gathers visited[w])
    kDirPull = 2,      // pull over out-edges of vertices not yet visited by every frontier colour
};
constexpr uint32_t kPullMaxWords = 8;  // pull levels need WB <= 8 (dense frontier rows)
constexpr int kPolicyIn = 6, kPolicyHidden = 32, kPolicyOut = 8;
// outputs 5..7 of the policy network rank these row widths (words)
constexpr uint32_t kPolicyWidthOut = 5, kPolicyWidthCount = 3;
constexpr uint32_t kPolicyWidths[kPolicyWidthCount] = {4, 16, 64};
constexpr int kPolicyParams = kPolicyIn * kPolicyHidden + kPolicyHidden + kPolicyHidden * kPolicyHidden +
                              kPolicyHidden + kPolicyHidden * kPolicyOut + kPolicyOut;

enum RefillMode : uint32_t {
    kRefillLane = 0,   // a colour lane takes the next sample as soon as its traversal ends
    kRefillBatch = 1,  // lanes are refilled only when every lane of the row has finished
};

// Device-resident control block of one sampling run.  Written and read only
// by the engine's kernels (and by the host between runs).
struct Ctl {
    // The counters that kernels take returned atomics on (the expand's chunk
    // counters and pending count, the commit's allocation counters) each start
    // a 128-byte line of their own, apart from the statistics and the fields
    // that all CTAs reduce into: a returned atomic or a load queues behind the
    // reductions on its line.
    alignas(128) unsigned int pend_count;  // vertices whose next row changed this level
    alignas(128) unsigned int chunk_next;  // expand's dynamic chunk counter
    alignas(128) unsigned long long new_packed;  // commit's allocation counter (units | groups << 26)
    alignas(128) unsigned long long list_count;  // frontier units for the coming expand
    unsigned long long list_groups;  // their total 4-edge groups
    unsigned int running;            // loop condition
    unsigned int host_flag[2];       // host mirror only: the loop condition after even / odd levels
    unsigned int error;              // ErrorBits
    unsigned int refill;             // RefillMode
    unsigned int bar_count, bar_gen; // grid barrier of the persistent kernel
    unsigned int dir;                // Direction of the coming level
    unsigned int frontier_lanes;     // lanes with colours in the coming level's frontier
    unsigned int sched;              // fbpt_schedule of the run
    unsigned long long tick, tick_limit;
    unsigned long long next_j, S;    // next sample index to hand out; samples in the run
    unsigned long long pair_cursor, pair_cap; // staging entries handed to finished samples' rows; capacity
    unsigned long long run_w[kMaxWords];   // lanes holding a sample
    unsigned long long act_w[kMaxWords];   // lanes present in the new frontier
    unsigned long long init_w[kMaxWords];  // lanes given a sample at the last schedule (init input)
    unsigned long long still_w[kMaxWords]; // lanes with colours in the current frontier
    alignas(16) unsigned int lane_j[kMaxLanes];        // sample index held by each lane
    alignas(16) unsigned int lane_cnt[kMaxLanes];      // RR entries of the lane's current sample so far
    unsigned int retired_j[kMaxLanes];     // sample index a finished lane held
    unsigned long long lane_base[kMaxLanes]; // staging position of a finished lane's row
    // sweep input, written by the schedule: finished lanes and the prefix of
    // their segment entry counts
    unsigned int fin_count;
    unsigned int fin_lane[kMaxLanes];
    unsigned int fin_pre[kMaxLanes + 1];
    unsigned long long fin_mask[kMaxWords]; // finished lanes as a bitmap (spill-log sweep)
    unsigned int spill_cur, spill_sweep;   // spill log buffer commit appends to; sweep it this level
    unsigned long long spill_len[2];
    unsigned long long sweep_work;   // entries the coming sweep reads (segments or spill log, the larger)
    // counters
    alignas(128) unsigned long long st_edges;
    unsigned long long st_calls, st_units, st_cev, st_assigned, st_push, st_pull, st_mask_words;
    unsigned long long st_groups;
    unsigned long long new_colours, list_colours;  // colour bits of the new / current frontier units
    // wide units: the commit's allocation counter (units | chunks << 26) and
    // their groups; the coming expand's units, chunks and groups; its chunk counter
    alignas(128) unsigned long long wide_packed;
    alignas(128) unsigned long long wide_gnew;
    unsigned long long wide_units, wide_chunks, wide_groups;
    alignas(128) unsigned int wchunk_next;
    unsigned int wpad;
    unsigned long long wide_need;  // largest wide-chunk count a level asked for beyond the capacity
    // compaction of the coming level (fbpt_compaction); stage rows the scan
    // commit has handed out
    unsigned int mode;
    alignas(128) unsigned int scan_rows;
    // phase times: first CTA start .. last CTA end of each phase (%globaltimer, ns);
    // index 0 expand, 1 commit, 2 sweep
    alignas(128) unsigned long long ph_t0[3], ph_t1[3], st_phase_ns[3];
};

// Per-graph, per-shape working memory.  Every array is all-zero between runs
// (the kernels restore what they dirty), except the scratch lists.
struct Workspace {
    uint32_t n = 0;
    uint32_t WB = 0;
    bool unfused = false;
    uint64_t* visited = nullptr;  // n * WB: colours that reached v
    uint64_t* next = nullptr;     // n * WB: colours reaching v at the current level
    uint64_t* nocc = nullptr;     // n: bit i set iff next[v][i] != 0 (and v is pending)
    uint64_t* stage = nullptr;    // pend_cap * WB: new frontier masks by pend index
    uint32_t* pend_v = nullptr;   // pend_cap
    uint32_t* seg = nullptr;      // 64 * WB * seg_cap: each lane's RR vertices
    uint32_t seg_cap = 0;         // entries per lane segment (a power of two >= kSegMin)
    uint64_t* spill = nullptr;    // 2 * spill_cap: (lane << 32 | vertex) beyond a full segment
    uint32_t* list_v = nullptr;   // list_cap
    uint32_t* list_mrow = nullptr;
    uint32_t* list_only = nullptr;
    uint64_t* list_rs = nullptr;
    uint64_t* list_re = nullptr;
    uint64_t* list_g = nullptr;
    uint64_t* list_occ = nullptr;
    uint32_t* chunk_u0 = nullptr; // chunk_cap
    uint4* wide_rec = nullptr;    // 2 * list_cap: wide unit records (32 B each)
    uint32_t* wide_chunk = nullptr; // wide_chunk_cap: unit of each wide chunk
    uint64_t wide_chunk_cap = 0;
    uint64_t* frontd = nullptr;   // n * WB when pull levels are allowed: frontier rows by vertex
    uint32_t* fstamp = nullptr;   // n: level whose frontier frontd[v] holds
    uint64_t pend_cap = 0, list_cap = 0, chunk_cap = 0, spill_cap = 0;
    Ctl* ctl = nullptr;
    Ctl* ctl_host = nullptr;      // pinned mirror
    bool clean = false;
    size_t bytes = 0;
};

// Kernel parameters of one run (passed by value).
struct Eng {
    uint32_t key0[10], key1[10];  // Philox round keys of seed (k0 + r * W0, k1 + r * W1), set by the host
    uint32_t n, WB;
    const uint64_t* row_ptr;
    const uint32_t* col;
    const uint32_t* thr;
    uint64_t seed, first_id, S;
    uint64_t* visited;
    uint64_t* next;
    uint64_t* nocc;
    uint64_t* stage;
    uint32_t* pend_v;
    uint32_t* seg;
    uint32_t seg_cap;
    uint64_t* spill;
    uint32_t* list_v;
    uint32_t* list_mrow;
    uint32_t* list_only;
    uint64_t* list_rs;
    uint64_t* list_re;
    uint64_t* list_g;
    uint64_t* list_occ;
    uint32_t* chunk_u0;
    // wide unit u: wide_rec[2u] = (first group lo, hi, colour words lo, hi),
    // wide_rec[2u + 1] = (groups, first chunk, stage row, edge masks: bits 0-3
    // the in-row edges of the first group, 4-7 those of the last)
    uint4* wide_rec;
    uint32_t* wide_chunk;
    uint64_t wide_chunk_cap;
    const uint64_t* orow;         // out-edge CSR (pull)
    const uint32_t* odst;
    const uint32_t* oeid;
    uint64_t* frontd;
    uint32_t* fstamp;
    const float* policy;          // kPolicyParams weights of the schedule network, or NULL
    const uint64_t* wpre;         // LT: exclusive prefix of the edge weights (m + 1)
    uint32_t model;               // fbpt_model
    uint32_t compaction;          // fbpt_compaction of fixed schedules
    uint64_t m;
    uint64_t pend_cap, list_cap, chunk_cap, spill_cap;
    uint32_t unfused;
    uint32_t alt;                 // levels may expand other than by plain push (launch k_expand_alt)
    Ctl* ctl;
    uint32_t* starts;             // S
    uint32_t* vcount;             // n
    uint32_t* rows_v;             // pair_cap: each finished sample's RR vertices, contiguous, unsorted
    uint64_t* row_start;          // S: staging position of sample index j's row
    uint32_t* row_len;            // S: its length
    fbpt_trace_row* trace;        // device copy of the per-level trace (NULL = off)
    uint64_t trace_cap;
    unsigned long long cond;      // cudaGraphConditionalHandle (0 = host-driven loop)
    uint32_t gated;               // host loop: the level kernels return at once when the run has ended
    uint32_t gated_pad;
    unsigned long long spin_limit;  // bounded waits of the persistent kernel's grid barrier
    // vertex order: rows of vertex label w are [rstart[w], rend[w]) (row_ptr and
    // row_ptr + 1 for the identity); perm maps a start vertex to its label and
    // inv a label back (NULL for the identity); order[k] is the sample index
    // the k-th refilled lane takes (NULL: k itself)
    const uint64_t* rstart;
    const uint64_t* rend;
    const uint32_t* perm;
    const uint32_t* inv;
    const uint32_t* order;
};

}  // namespace fbpt

// The opaque handle behind fbpt_policy*: the schedule network's parameters
// (input mean and scale, then the three layers), on the device and the host.
struct fbpt_policy {
    float* d_params = nullptr;
    float h_params[2 * fbpt::kPolicyIn + fbpt::kPolicyParams] = {};
};

// The opaque handle behind fbpt_graph*.
struct fbpt_graph {
    uint32_t n = 0;
    uint64_t m = 0;
    uint64_t* row_ptr = nullptr;  // n + 1
    uint32_t* col = nullptr;      // padded to a multiple of 4 (+4)
    uint32_t* thr = nullptr;
    cudaStream_t stream = nullptr;
    int device = 0;
    // out-edge CSR for pull levels, built on first use: out-row w lists
    // (v, e) for every in-edge e = (w -> v)
    uint64_t* orow = nullptr;     // n + 1
    uint32_t* odst = nullptr;     // m
    uint32_t* oeid = nullptr;     // m (edge ids < 2^32)
    uint64_t* wpre = nullptr;     // m + 1: exclusive prefix of the LT weights (units of 2^-32), built on first use
    int lt_rows = 0;              // 1: every row's LT weights sum to at most 1; -1: some row's exceed it
    fbpt::Workspace* ws = nullptr;
    double rr_hint = 32.0;        // running estimate of RR entries per sample
    fbpt_tuning tuned = {};       // launch shape measured by fbpt_autotune
    bool tuned_valid = false;
    // vertex order (fbpt_graph_set_order); all NULL for the identity
    uint32_t* perm = nullptr;     // n: new label of each vertex
    uint32_t* inv = nullptr;      // n: vertex of each new label
    uint32_t* col0 = nullptr;     // m: the caller's sources (col then holds perm[col0])
    uint64_t* rstart = nullptr;   // n: in-row start of each new label (row_ptr[inv[v']])
    uint64_t* rend = nullptr;     // n: its end (row_ptr[inv[v'] + 1])
    uint32_t sorted_starts = 0;   // samples take lanes by increasing (relabelled) start vertex
};

namespace fbpt {
int workspace_release(fbpt_graph* g);
int sample_impl(fbpt_graph* g, uint64_t seed, uint64_t first_id, uint64_t S, const fbpt_opts* opts, fbpt_rrsets* out,
                fbpt_stats* stats);
int sample_batched_impl(uint32_t G, fbpt_graph* const* gs, const uint64_t* seeds, const uint64_t* first_ids,
                        const uint64_t* Ss, const fbpt_opts* opts, fbpt_rrsets* outs, fbpt_stats* stats);
int autotune_impl(fbpt_graph* g, uint64_t seed, uint64_t S, const fbpt_opts* base, fbpt_tuning* out);
int policy_width_impl(fbpt_graph* g, uint64_t seed, uint64_t S, const fbpt_opts* base, uint32_t* row_words,
                      float* scores);
int imm_impl(fbpt_graph* g, uint32_t k, double epsilon, double ell, uint64_t seed, uint64_t max_samples,
             const fbpt_opts* opts, uint32_t* seeds_host, uint64_t* gains_host, fbpt_imm_result* result,
             fbpt_stats* stats);
// Builds g's out-edge CSR if it is not there yet (FBPT_EUNSUPPORTED for m >= 2^32).
int ensure_out_csr(fbpt_graph* g, cudaStream_t st);
// Builds g's LT weight prefix if it is not there yet; FBPT_EINVAL if a row's weights exceed 1.
int ensure_lt_weights(fbpt_graph* g, cudaStream_t st);
// Device-wide exclusive scan of n counts into n+1 uint64 offsets (out[n] = total).
int exclusive_scan_u32(const uint32_t* in, uint64_t* out, uint64_t n, cudaStream_t st);
int exclusive_scan_u64(const uint64_t* in, uint64_t* out, uint64_t n, cudaStream_t st);
// Stable LSD radix sort of n 64-bit keys on their low `bits` bits (tmp: n scratch keys).
int radix_sort_u64(uint64_t* keys, uint64_t* tmp, uint64_t n, uint32_t bits, cudaStream_t st);
// Device array order[S]: sample indices 0 .. S-1 by increasing (relabelled)
// start vertex, ties by index (g->sorted_starts); caller frees with cudaFreeAsync.
int start_order(const fbpt_graph* g, uint64_t seed, uint64_t first_id, uint64_t S, cudaStream_t st,
                uint32_t** order);
// Places fbpt_select_seeds_noalloc's fixed scratch array on the current device
// (its module is loaded on first use; graph creation calls this).
int noalloc_preload();
}  // namespace fbpt
