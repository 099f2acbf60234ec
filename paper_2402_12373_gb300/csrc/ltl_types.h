// ltl_types.h -- plain structs shared by the host driver and the kernels.
#pragma once
#include <cstdint>

namespace ltl {

// Connectives (and atoms) as stored in provenance words and programs.
enum Op : int { OP_ATOM = 0, OP_NOT = 1, OP_AND = 2, OP_OR = 3, OP_X = 4, OP_F = 5, OP_G = 6, OP_U = 7 };

constexpr int kMaxLevels = 64;
constexpr uint64_t kValPending = 0xFFFFFFFFull;   // slot claimed, entry not yet published
constexpr uint64_t kValFail = 0xFFFFFFFEull;      // slot claimed but the cache was full

// One slot of the device hash set: the fingerprint key (0 = empty) and the
// entry index (or kValPending / kValFail), read and written together by
// 128-bit atomics, so that the claim of a slot also returns the index an
// earlier claimant published there.
struct alignas(16) HSlot {
    unsigned long long key;
    unsigned long long val;
};
constexpr uint64_t kMaxEntries = (1ull << 30) - 1;

// Cache admission policies (relaxed uniqueness checks, Section 5).
enum Ruc : uint32_t { RUC_EXACT = 0, RUC_HASH = 1, RUC_FKP = 2 };
constexpr uint64_t kKey63 = (1ull << 63) - 1;   // relaxed admission keys have 63 bits

// Provenance of a cache entry, packed: op in bits 60..62, left operand (or the
// proposition index of an atom) in bits 30..59, right operand in bits 0..29.
__host__ __device__ inline uint64_t prov_pack(int op, uint64_t a, uint64_t b) {
    return ((uint64_t)op << 60) | (a << 30) | b;
}
__host__ __device__ inline int prov_op(uint64_t p) { return (int)(p >> 60); }
__host__ __device__ inline uint64_t prov_a(uint64_t p) { return (p >> 30) & ((1ull << 30) - 1); }
__host__ __device__ inline uint64_t prov_b(uint64_t p) { return p & ((1ull << 30) - 1); }

// Candidate tiles: rectangular tiles of up to kTileA x kTileB (left x right
// operand) pairs; unary segments are cut into runs of up to kTileU operands.
// The host shrinks tiles when a launch has few candidates, so that every
// resident CTA gets work.
constexpr int kTileA = 8;
constexpr int kTileB = 8;
constexpr int kTileU = 16;

enum SegKind : int { SEG_UNARY = 0, SEG_RECT = 1, SEG_TRI = 2 };

// One (connective, split) part of a size level's candidate space.
struct Seg {
    int32_t op;            // Op
    int32_t kind;          // SegKind
    uint64_t a_begin;      // first left operand (cache index; proposition for atoms)
    uint64_t a_count;
    uint64_t b_begin;      // first right operand (binary only)
    uint64_t b_count;
    uint64_t tile_begin;   // first tile id of this segment within the level
    uint64_t n_tiles;
    uint32_t n_ta, n_tb;   // tiles along a and along b
    int32_t a_inner;       // RECT: 1 = a-tile index varies fastest
    uint32_t ta, tb;       // tile extent along a (unary: run length) and along b
    int32_t prob;          // index of the problem (engine slot) the segment belongs to
    int32_t level;         // size level the candidates have
};

// Device control block (one per learn call).
struct Ctrl {
    unsigned long long n_entries;      // bump pointer of the cache arena
    unsigned long long cands;          // candidates processed (cumulative)
    unsigned long long compares;       // full-matrix compares after fingerprint match
    unsigned long long collisions;     // compares that found a different matrix
    unsigned int found_count;          // separators seen (first one is recorded)
    int stop;                          // 1: CTAs leave at the next tile boundary
    int cap_hit;
    int err;                           // 0 or an ltl_status error code
    unsigned long long found_prov;     // provenance of the recorded separator
    int found_level;
    int invalid_letter;                // set by the packer on a letter >= 2^n_props
    unsigned long long timeouts;
};

// Device view of one learning problem.
struct Problem {
    uint64_t *arena;              // entries x stride words
    uint64_t stride;              // words per characteristic matrix = W * plane
    uint64_t plane;               // padded trace count (words per bit-plane)
    const uint64_t *mask;         // W planes: positions < length
    const uint64_t *keys;         // W planes: NH keys
    const uint64_t *atoms;        // n_props matrices (level-1 sources)
    uint64_t *prov;               // packed provenance per entry
    HSlot *hslots;                // hash slots (all zero = empty)
    uint64_t hmask;               // slots - 1
    uint64_t max_entries;
    Ctrl *ctrl;
    uint32_t n_traces;            // real traces (|P| + |N|)
    uint32_t n_pos;               // positives are traces [0, n_pos)
    int32_t nsteps;               // log-step count: ceil(log2(max length))
    uint32_t logstep;             // F, G, U by the log-step exponential propagation
                                  // (Section 4); 0: by the carry chain
    int32_t stop_first;           // stop at the first separator
    uint32_t groups;              // chunk groups per matrix (1: kept in registers)
    uint32_t max_errors;          // misclassified traces a separator may have
    uint32_t ruc;                 // admission policy: RUC_EXACT, RUC_HASH, RUC_FKP
    uint32_t fkp_b;               // RUC_FKP: leading positions taken per trace
    uint64_t key_mask;            // relaxed modes: admission-key bits kept (63 or fewer)
    unsigned long long spin_limit;
};

// Extent of a launch whose level was planned on the device.
struct LevelDesc {
    int32_t n_segs;
    int32_t pad;
    uint64_t total_tiles;
};

// One launch: the segments of one connective for every problem of one launch
// shape, each problem at its own size level.
struct LevelArgs {
    const Seg *segs;
    const Problem *probs;              // problem descriptors, indexed by Seg::prob
    unsigned long long *tile_counter;  // this launch's tile counter (zeroed before)
    int32_t n_segs;
    int32_t pad;
    uint64_t total_tiles;
    const LevelDesc *desc;             // non-null: n_segs and total_tiles come from here
    unsigned long long *staged;        // non-null: operand matrices the launch copied
                                       // into shared memory are added here (fused kernel)
};

// One formula reconstruction: the provenance array of a problem, its entry
// count, and the provenance word of the root (a cache entry or a separator).
struct WalkJob {
    const uint64_t *prov;
    uint64_t n_entries;
    uint64_t root;
};

}  // namespace ltl
