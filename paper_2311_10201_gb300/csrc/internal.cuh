// Internal structures of libfbpt shared by its translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace fbpt {

constexpr uint32_t kMaxWords = 64;      // words per vertex row (slots * W)
constexpr uint32_t kMaxSlots = 64;
constexpr uint32_t kUnitBits = 26;      // list allocation counter: units in the low 26 bits
constexpr uint64_t kUnitMask = (1ull << kUnitBits) - 1;
constexpr uint32_t kTileGroups = 1024;  // edge groups (4 edges each) per expand tile

enum SlotState : uint32_t { kSlotIdle = 0, kSlotRunning = 1 };

enum ErrorBits : uint32_t {
    kErrListOverflow = 1u,
    kErrTileOverflow = 2u,
    kErrTickLimit = 4u,
    kErrPendOverflow = 8u,
};

// Device-resident control block of one sampling run.  Written and read only
// by the engine's kernels (and by the host between runs).
struct Ctl {
    unsigned long long list_count;   // frontier units for the coming expand
    unsigned long long list_groups;  // their total 4-edge groups
    unsigned long long new_packed;   // commit's allocation counter (units | groups << 26)
    unsigned long long active_mask;  // slots with a unit in the new list
    unsigned int pend_count;         // vertices whose next mask changed this level
    unsigned int tile_next;          // expand's dynamic tile counter
    unsigned int running;            // loop condition
    unsigned int fin_count;
    unsigned int init_count;
    unsigned int error;              // ErrorBits
    unsigned long long tick, tick_limit;
    unsigned long long next_batch, nbatches;
    unsigned long long pair_cursor, pair_cap;
    unsigned int slot_state[kMaxSlots];
    unsigned int slot_ncol[kMaxSlots];
    unsigned long long slot_base[kMaxSlots];  // sample id of colour 0 of the slot's batch
    unsigned int tcount[kMaxSlots];           // touched vertices of the slot's batch
    unsigned int fin_slot[kMaxSlots];
    unsigned int fin_ncol[kMaxSlots];
    unsigned long long fin_base[kMaxSlots];
    unsigned int init_slot[kMaxSlots];
    // counters
    unsigned long long st_edges, st_calls, st_units, st_cev, st_batches, st_push, st_pull;
    // expand kernel time: first CTA start .. last CTA end of each launch (%globaltimer, ns)
    unsigned long long exp_t0, exp_t1, st_expand_ns, st_mask_words;
};

// Per-graph, per-shape working memory.  Every array is all-zero between runs
// (the kernels restore what they dirty), except the scratch lists.
struct Workspace {
    uint32_t n = 0;
    uint32_t W = 0, B = 0, WB = 0;
    uint64_t nw = 0;              // 64-bit words of an n-bit bitmap
    uint64_t* visited = nullptr;  // n * WB
    uint64_t* next = nullptr;     // n * WB
    uint64_t* stage = nullptr;    // pend_cap * WB: new frontier masks by pend index
    uint64_t* dirty = nullptr;    // nw
    uint64_t* touched = nullptr;  // B * nw
    uint32_t* tlist = nullptr;    // B * n
    uint32_t* pend_v = nullptr;   // pend_cap
    uint32_t* list_v = nullptr;   // list_cap
    uint32_t* list_mrow = nullptr;
    uint32_t* list_only = nullptr;
    uint64_t* list_g = nullptr;
    uint64_t* list_occ = nullptr;
    uint32_t* tile_u0 = nullptr;  // tile_cap
    uint64_t pend_cap = 0, list_cap = 0, tile_cap = 0;
    bool unfused = false;
    Ctl* ctl = nullptr;
    Ctl* ctl_host = nullptr;      // pinned mirror
    bool clean = false;
    size_t bytes = 0;
};

// Kernel parameters of one run (passed by value).
struct Eng {
    uint32_t n, W, B, WB;
    uint64_t nw;
    const uint64_t* row_ptr;
    const uint32_t* col;
    const uint32_t* thr;
    uint64_t seed, first_id, S;
    uint64_t* visited;
    uint64_t* next;
    uint64_t* stage;
    uint64_t* dirty;
    uint64_t* touched;
    uint32_t* tlist;
    uint32_t* pend_v;
    uint32_t* list_v;
    uint32_t* list_mrow;
    uint32_t* list_only;
    uint64_t* list_g;
    uint64_t* list_occ;
    uint32_t* tile_u0;
    uint64_t pend_cap, list_cap, tile_cap;
    uint32_t unfused;
    uint32_t vbits;               // bits of a vertex id in a pair key
    Ctl* ctl;
    uint32_t* starts;             // S
    uint32_t* vcount;             // n
    uint64_t* pairs;              // pair_cap: (sample index << vbits) | vertex
    unsigned long long cond;      // cudaGraphConditionalHandle (0 = host-driven loop)
};

}  // namespace fbpt

// The opaque handle behind fbpt_graph*.
struct fbpt_graph {
    uint32_t n = 0;
    uint64_t m = 0;
    uint64_t* row_ptr = nullptr;  // n + 1
    uint32_t* col = nullptr;      // padded to a multiple of 4 (+4)
    uint32_t* thr = nullptr;
    cudaStream_t stream = nullptr;
    int device = 0;
    fbpt::Workspace* ws = nullptr;
    double rr_hint = 32.0;        // running estimate of RR entries per sample
};

namespace fbpt {
int workspace_release(fbpt_graph* g);
// Device-wide exclusive scan of n counts into n+1 uint64 offsets (out[n] = total).
int exclusive_scan_u32(const uint32_t* in, uint64_t* out, uint64_t n, cudaStream_t st);
int exclusive_scan_u64(const uint64_t* in, uint64_t* out, uint64_t n, cudaStream_t st);
// Stable LSD radix sort of 64-bit keys on their low `bits` bits; `tmp` holds n keys.
// The result ends in `keys`.
int radix_sort_u64(uint64_t* keys, uint64_t* tmp, uint64_t n, uint32_t bits, cudaStream_t st);
}  // namespace fbpt
