// ltl_engine.cu -- the host engine: problems resident in a device workspace,
// advanced size level by size level in rounds (Section 3, `enum`).
//
// One round = for every resident problem, the candidate space of its next
// size level (the segments of Section 3's handleOp: one connective and one
// split each), grouped by launch shape and connective; one persistent launch
// per group pulls tiles from any of its problems.  After the round the
// control blocks of all problems are read back at once, levels are closed,
// finished problems get their formula rebuilt (one batched provenance walk)
// and release their memory, and waiting problems are admitted.
//
// ltl_ctx_* drive one problem at a time through an engine; ltl_learn_batch
// and the server drive many.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <deque>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <set>
#include <thread>
#include <tuple>
#include <vector>

#include "ltl_autotune.h"
#include "ltl_internal.h"
#include "ltl_plan.h"

namespace ltl {
namespace {

constexpr uint64_t kKeySeed = 0x243F6A8885A308D3ull;   // NH key stream seed (digits of pi)
constexpr int kMaxTokens = 256;
constexpr int kMaxGroups = 512;                       // launches per round
// Rounds with fewer candidates than this run their launches concurrently on
// auxiliary streams: small levels are launch-latency bound, and the
// connectives of a level are independent (they meet only in the lock-free
// hash set).  Larger rounds run their launches one after another, so each
// launch's time is its own.
constexpr uint64_t kConcurrentBelow = 1ull << 17;
// host-planned rounds of one problem below this many candidates run their launches concurrently
constexpr uint64_t kRoundConcurrentBelow = 1ull << 18;
constexpr int kAuxStreams = 8;
// A chain of device-planned levels becomes a CUDA graph the eighth time its
// shape is enqueued; up to this many shapes are kept.
constexpr int kChainCaptureAfter = 8;
constexpr size_t kChainShapes = 256;

// Where one problem's device state lives, relative to its region base.
struct Layout {
    int W = 0, Wt = 0, C = 0, NT = 0, NB = 1;
    int block = 0;          // threads per CTA: NT, plus the hash warps of the warp-specialised kernel
    int CL = 0;             // CTAs per cluster of the cluster kernel (0: not used)
    bool narrow = false;
    bool ws = false;        // warp-specialised level kernel for every launch (on request)
    bool ws_ok = false;     // the warp-specialised kernel exists for this shape and its ring fits
    size_t ws_smem = 0;     // its dynamic shared memory
    size_t stream_smem = 0; // the streaming kernel's operand ring (matrices larger than one CTA)
    uint32_t G = 0;
    uint32_t n_traces = 0, n_pos = 0;
    int n_props = 0, nsteps = 0;
    uint64_t plane = 0, stride = 0;
    uint64_t hslots = 0, max_entries = 0;
    size_t smem = 0;
    size_t o_letters, o_offsets, o_mask, o_keys, o_atoms, o_hslots, o_prov, o_arena, end;
};

// Everything the engine needs to know about one problem's input.
struct ProblemIn {
    // host input: positives and negatives (engine-owned copies when `own`)
    const uint32_t *hl[2] = {nullptr, nullptr};
    const uint64_t *ho[2] = {nullptr, nullptr};
    uint64_t hn[2] = {0, 0};
    std::unique_ptr<uint32_t[]> own_l[2];
    std::unique_ptr<uint64_t[]> own_o[2];
    // device input: positives then negatives, one offset array
    const uint32_t *d_letters = nullptr;
    const uint64_t *d_offsets = nullptr;
    bool device_input = false;
    uint64_t n_pos = 0, n_neg = 0, max_len = 0, total_pos = 0;
    int n_props = 1;
    uint32_t ops = LTL_ALL;
    int max_size = 1;
    uint64_t budget = 0;
    uint64_t id = 0;
    double t_submit = 0;
};

enum SlotState { SLOT_FREE = 0, SLOT_RUNNING = 1, SLOT_DONE = 2 };

struct Slot {
    int state = SLOT_FREE;
    ProblemIn in;
    Layout L;
    size_t off = 0, bytes = 0;   // region in the workspace
    int level = 1;               // next size level to enumerate
    uint64_t lvl_begin[kMaxLevels] = {}, lvl_count[kMaxLevels] = {};
    uint64_t prev_entries = 0, prev_cands = 0;
    bool found = false;
    ltl_status status = LTL_NOT_FOUND;
    std::string formula;
    std::string error;
    ltl_stats st;
    uint32_t rounds = 0;
    double t_admit = 0, t_done = 0;
};

// First-fit allocator over byte offsets of the workspace.
struct FreeList {
    std::map<size_t, size_t> free;   // offset -> size
    void reset(size_t begin, size_t end) {
        free.clear();
        if (end > begin) free[begin] = end - begin;
    }
    bool alloc(size_t bytes, size_t &off) {
        for (auto it = free.begin(); it != free.end(); ++it) {
            if (it->second >= bytes) {
                off = it->first;
                const size_t rest = it->second - bytes;
                free.erase(it);
                if (rest) free[off + bytes] = rest;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        auto it = free.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free.erase(nx);
        }
        if (it != free.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free.erase(it);
            }
        }
    }
    size_t largest() const {
        size_t m = 0;
        for (const auto &kv : free) m = std::max(m, kv.second);
        return m;
    }
};

// Chooses the launch shape of a problem and carves its region for `budget`
// bytes (0: as many entries as `avail` bytes allow).
// Dynamic shared memory the warp-specialised kernel may take: what is left
// of the opt-in maximum (227 KB) after its static part, rounded down.
constexpr size_t kWsSmemMax = 224 * 1024;
// A problem's round of at least this many candidates runs the
// warp-specialised kernel under LTL_KERNEL_AUTO (when its shape has one).
constexpr uint64_t kWsAutoMin = 1ull << 15;

// Page-locked host blocks outlive the engines that use them.  Pinning costs
// tens of microseconds per call plus time per page (the 64 MiB staging buffer
// milliseconds), more than a small ltl_learn_batch call's own work, and every
// such call builds an engine of its own.  So a block an engine releases goes
// to the free list of its size class (powers of two from 4 KiB) and the next
// engine takes it from there; blocks are never returned to the driver, so the
// cache holds at most what the engines alive at one time held.  An engine
// releases its blocks only after synchronising the stream their copies ran on.
class PinnedCache {
public:
    static PinnedCache &get() {
        static PinnedCache *c = new PinnedCache();
        return *c;
    }
    cudaError_t alloc(void **p, size_t bytes) {
        const int cls = size_class(bytes);
        {
            std::lock_guard<std::mutex> lk(mu);
            std::vector<void *> &fl = free_list[cls];
            if (!fl.empty()) {
                *p = fl.back();
                fl.pop_back();
                return cudaSuccess;
            }
        }
        const cudaError_t e = cudaMallocHost(p, (size_t)1 << cls);
        if (e == cudaSuccess) {
            std::lock_guard<std::mutex> lk(mu);
            class_of[*p] = cls;
        }
        return e;
    }
    void release(void *p) {
        if (!p) return;
        std::lock_guard<std::mutex> lk(mu);
        const auto it = class_of.find(p);
        if (it == class_of.end()) {
            cudaFreeHost(p);   // not a block of this cache
            return;
        }
        free_list[it->second].push_back(p);
    }

private:
    static int size_class(size_t bytes) {
        int c = 12;
        while (((size_t)1 << c) < bytes) ++c;
        return c;
    }
    std::mutex mu;
    std::map<void *, int> class_of;
    std::vector<void *> free_list[64];
};

template <class T>
cudaError_t pinned_alloc(T **p, size_t bytes) {
    void *v = nullptr;
    const cudaError_t e = PinnedCache::get().alloc(&v, bytes);
    *p = (T *)v;
    return e;
}

// Launch properties of the level kernels, shared by every engine of the
// process: the opt-in to the device's shared-memory maximum, the carveout and
// the permission for clusters of more than 8 CTAs are attributes of the
// function, and the resident CTAs (or clusters) depend only on the function,
// block size, shared memory, cluster size and device.  Queried again in every
// engine they cost each ltl_learn_batch call (an engine of its own) tens of
// CUDA calls.
struct LaunchCache {
    static LaunchCache &get() {
        static LaunchCache *c = new LaunchCache();
        return *c;
    }
    std::mutex mu;
    std::map<std::tuple<int, const void *, int, size_t>, int> occ;           // resident CTAs per SM
    std::map<std::pair<int, const void *>, int> dyn_max;                     // opted in: its dynamic smem maximum
    std::set<std::pair<int, const void *>> nonportable;                      // clusters of 16 allowed
    std::map<std::tuple<int, const void *, int, size_t, int>, int> clusters;   // resident clusters
};

// Shared memory one CTA of the cluster kernel may hold its slice in.
constexpr size_t kClusterSliceMax = 200 * 1024;

ltl_status plan_layout(const ProblemIn &in, uint32_t max_chunks, uint32_t level_kernel, uint64_t budget,
                       uint64_t avail, Layout &L) {
    const uint64_t T = in.n_pos + in.n_neg;
    if (T > 0x7fffffffull) return fail(LTL_ERR_INVALID, "too many traces (%llu)", (unsigned long long)T);
    L = Layout{};
    L.n_traces = (uint32_t)T;
    L.n_pos = (uint32_t)in.n_pos;
    L.n_props = in.n_props;
    L.W = (int)std::max<uint64_t>(1, (in.max_len + 63) / 64);
    L.Wt = (int)pow2_ceil((uint64_t)L.W);
    if (L.Wt > 8) return fail(LTL_ERR_INVALID, "traces longer than 512 positions are not supported by ltl_learn");
    L.nsteps = ceil_log2(in.max_len);
    // Each thread holds C pairs of words (C * W <= 8) of a candidate; a CTA of
    // up to 256 threads holds a whole matrix (fused kernel); larger matrices
    // go through the two-pass streaming kernel in `G` chunk groups.  The
    // narrow layout packs two traces of <= 32 positions per word.
    const int Cmax = 8 / L.Wt;
    const uint64_t maxNT = 256;
    const uint64_t pairs = std::max<uint64_t>(1, (T + 1) / 2);
    const uint64_t quads = std::max<uint64_t>(1, (T + 3) / 4);
    const uint64_t cap_c = max_chunks ? pow2_ceil(max_chunks) : 8;
    const uint64_t ncmax = std::min<uint64_t>(4, cap_c);
    auto shape = [&](uint64_t units, uint64_t cmax) {
        uint64_t nt = pow2_ceil((units + cmax - 1) / cmax);
        nt = std::min<uint64_t>(std::max<uint64_t>(nt, 32), maxNT);
        L.NT = (int)nt;
        L.C = (int)std::min<uint64_t>(pow2_ceil((units + nt - 1) / nt), cmax);
        L.G = 1;
    };
    if (in.max_len <= 32 && quads <= maxNT * ncmax) {
        shape(quads, ncmax);
        L.narrow = true;
    } else if (pairs <= maxNT * std::min<uint64_t>(Cmax, cap_c)) {
        shape(pairs, std::min<uint64_t>(Cmax, cap_c));
    } else if (pairs <= maxNT * (uint64_t)Cmax) {
        shape(pairs, (uint64_t)Cmax);
    } else {
        // streaming: CTAs of 128 threads (two resident per SM where 256 fit
        // one; measured 3-6 % faster on the 65,536-trace workload)
        const uint64_t snt = 128;
        L.NT = (int)snt;
        L.C = Cmax;
        L.G = (uint32_t)((pairs + snt * Cmax - 1) / (snt * Cmax));
    }
    // Matrices larger than one CTA: a cluster of CL CTAs (a power of two, at
    // most 8, or 16 when 8 slices would not fit shared memory) holds one
    // candidate in shared memory, one slice of whole chunk groups per CTA; the
    // chunk groups are padded to a multiple of CL.  When no cluster fits, the
    // two-pass streaming kernel runs instead.
    if (L.G >= 2 && cluster_kernel_ptr(L.Wt, L.C) && level_kernel != LTL_KERNEL_FUSED) {
        auto slice_bytes = [&](uint32_t cl) {
            const uint64_t g = (L.G + cl - 1) / cl * cl;
            return (uint64_t)L.Wt * (g / cl) * L.C * 2 * L.NT * 8;
        };
        uint32_t cl = 1;
        while (cl * 2 <= 8 && cl * 2 <= L.G) cl *= 2;
        if (slice_bytes(cl) > kClusterSliceMax && L.G >= 16) cl = 16;
        if (slice_bytes(cl) <= kClusterSliceMax) {
            L.CL = (int)cl;
            L.G = (L.G + cl - 1) / cl * cl;
        }
    }
    // the batch size the fused kernel of this shape was compiled with (its
    // shared-memory operand slots are sized from it)
    L.NB = L.G == 1 ? fused_kernel_batch(L.Wt, L.C, L.narrow) : 1;
    if (L.G == 1 && L.NB < 1) return fail(LTL_ERR_INVALID, "no fused kernel for W=%d C=%d", L.Wt, L.C);
    L.plane = (uint64_t)L.G * L.C * 2 * L.NT;   // words per bit-plane
    L.stride = (uint64_t)L.Wt * L.plane;
    L.smem = L.G == 1 ? (size_t)(L.NB + 1) * 8 * L.stride : 0;
    if (L.CL) L.smem = (size_t)L.Wt * (L.plane / L.CL) * 8;   // the CTA's slice
    if (L.G > 1) L.stream_smem = stream_smem_bytes(L.Wt, L.C, L.NT);
    L.block = L.NT;
    // the warp-specialised kernel adds a ring of two batches of results (its
    // own compiled batch size)
    const int ws_nb = L.G == 1 ? ws_kernel_batch(L.Wt, L.C, L.narrow) : 1;
    const size_t ws_smem = (size_t)(3 * ws_nb + 1) * 8 * L.stride;
    L.ws_smem = ws_smem;
    L.ws_ok = L.G == 1 && ws_nb == L.NB && ws_smem <= kWsSmemMax;
    // on request, any shape whose ring fits, for every launch; the automatic
    // choice takes it per launch (large rounds, see round())
    const bool want_ws = level_kernel == LTL_KERNEL_WS;
    if (L.G == 1 && want_ws && ws_smem <= kWsSmemMax) {
        L.ws = true;
        L.NB = ws_nb;
        L.smem = ws_smem;
        L.block = L.NT + kWsExtraThreads;
    }

    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t r = o;
        o = round_up(o + bytes, 256);
        return r;
    };
    L.o_letters = take(in.device_input ? 0 : sizeof(uint32_t) * std::max<uint64_t>(in.total_pos, 1));
    L.o_offsets = take(in.device_input ? 0 : sizeof(uint64_t) * (T + 1));
    L.o_mask = take(8 * L.stride);
    L.o_keys = take(8 * L.stride);
    L.o_atoms = take(8 * L.stride * (uint64_t)in.n_props);
    const size_t fixed = o;
    const uint64_t total = budget ? budget + fixed : avail;
    if (total <= fixed + 4096) return fail(LTL_ERR_OOM, "memory too small for the problem layout");
    const uint64_t R = total - fixed - 4096;
    const uint64_t per = 8 * L.stride + 8;   // arena + provenance per entry
    const uint64_t sb = sizeof(HSlot);   // bytes per hash slot, two slots per entry
    uint64_t E = R / (per + 2 * sb);
    uint64_t slots = pow2_ceil(std::max<uint64_t>(2 * E, 1024));
    while (slots * sb + E * per > R && E > 0) {
        E = (R > slots * sb) ? (R - slots * sb) / per : 0;
        if (slots > 1024 && slots / 2 >= 2 * E) slots /= 2;
    }
    E = std::min<uint64_t>(E, kMaxEntries);
    if (E < 1) return fail(LTL_ERR_OOM, "memory too small for one cache entry");
    L.max_entries = E;
    L.hslots = slots;
    L.o_hslots = take(sizeof(HSlot) * slots);
    L.o_prov = take(8 * E);
    L.o_arena = take(8 * L.stride * E);
    L.end = o;
    return LTL_OK;
}

// Candidate space of cost level k of one problem, as segments tagged with the
// problem's slot and the level (the shared planner code of ltl_plan.h).
void level_segments(const Slot &s, int k, int prob, const Costs &cost, std::vector<Seg> &out) {
    auto emit = [&](Seg sg) {
        sg.prob = prob;
        sg.level = k;
        out.push_back(sg);
    };
    plan_level_segments(s.in.ops, s.in.n_props, s.lvl_begin, s.lvl_count, k, cost, emit);
}

}  // namespace

// ===================================================================== Engine

class Engine {
public:
    ltl_opts opts{};
    int device = 0, n_sm = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    char *ws = nullptr;
    size_t ws_bytes = 0;
    bool ws_owned = false;
    int max_slots = 1;
    bool keep_finished = false;   // contexts keep the last problem for introspection
    // shared region at the start of the workspace
    size_t o_probs = 0, o_ctrls = 0, o_segs = 0, o_counters = 0, o_jobs = 0, o_tokens = 0, o_ntok = 0, shared_end = 0;
    int probs_lo = INT32_MAX, probs_hi = -1;   // slots whose descriptors await upload
    size_t o_plan_state = 0, o_plan_log = 0, o_descs = 0;   // device planning of small levels
    PlanState *h_plan_state = nullptr;
    PlanLog *h_plan_log = nullptr;
    size_t max_segs = 0;
    Problem *h_probs = nullptr;
    Ctrl *h_ctrls = nullptr;
    unsigned long long *h_staged = nullptr;   // staged-operand counts of a round's launches
    Seg *h_segs = nullptr;
    WalkJob *h_jobs = nullptr;
    uint32_t *h_tokens = nullptr;
    int *h_ntok = nullptr;
    // Pinned staging of small host inputs: a problem's letters and offsets are
    // copied into this buffer and uploaded from it asynchronously (from
    // pageable memory each upload would wait for the stream); the buffer is
    // reused once the stream has drained.
    static constexpr size_t kPinStageMax = (size_t)4 << 20;     // inputs staged when at most this size
    static constexpr size_t kPinStageBytes = (size_t)64 << 20;
    char *h_pin = nullptr;
    size_t pin_head = 0;
    std::vector<Slot> slots;
    FreeList mem;
    cudaEvent_t ev_begin = nullptr, ev_end = nullptr;
    std::vector<cudaEvent_t> ev_op;   // after each launch of a round, created on demand
    std::vector<cudaEvent_t> ev_chain;   // device-planned chains: per level, its start and each launch
    std::map<std::string, cudaGraphExec_t> chain_graphs;   // captured chains by shape
    std::map<std::string, int> chain_seen;                  // times each uncaptured shape was enqueued
    cudaStream_t cap_stream = nullptr;   // stream chains are captured on
    std::vector<cudaStream_t> aux;    // concurrent launches of small rounds, created on demand
    Tuner tuner;                      // tile size and occupancy per launch class (when enabled)
    uint64_t total_rounds = 0;

    ~Engine() { teardown(); }

    ltl_status setup(const ltl_opts *o, int max_resident, bool keep) {
        opts = *o;
        // the caller's string need not outlive this call
        tuner.enabled = opts.autotune_path != nullptr;
        tuner.path = opts.autotune_path ? opts.autotune_path : "";
        opts.autotune_path = nullptr;
        tuner.load();
        if (opts.ruc > LTL_RUC_FKP) return fail(LTL_ERR_INVALID, "ruc must be LTL_RUC_EXACT, LTL_RUC_HASH or LTL_RUC_FKP");
        if (opts.ruc_mask_bits > 62) return fail(LTL_ERR_INVALID, "ruc_mask_bits must be at most 62");
        if (opts.level_kernel > LTL_KERNEL_WS) return fail(LTL_ERR_INVALID, "level_kernel must be LTL_KERNEL_AUTO, _FUSED or _WS");
        if (opts.level_planning > LTL_PLAN_HOST) return fail(LTL_ERR_INVALID, "level_planning must be LTL_PLAN_AUTO or _HOST");
        if (opts.propagation > LTL_PROP_LOGSTEP)
            return fail(LTL_ERR_INVALID, "propagation must be LTL_PROP_CARRY or LTL_PROP_LOGSTEP");
        keep_finished = keep;
        max_slots = std::max(1, std::min(max_resident, 4096));
        cudaError_t e = cudaGetDevice(&device);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, device);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            return fail(LTL_ERR_CUDA, "no usable CUDA device: %s", cudaGetErrorString(e));
        }
        if (opts.stream) stream = (cudaStream_t)opts.stream;
        else {
            LTL_CUDA_TRY(cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking));
            own_stream = true;
        }
        // shared region
        max_segs = (size_t)max_slots * 64 + 1024;
        size_t cur = 0;
        auto take = [&](size_t bytes) {
            const size_t r = cur;
            cur = round_up(cur + bytes, 256);
            return r;
        };
        o_probs = take(sizeof(Problem) * max_slots);
        o_ctrls = take(sizeof(Ctrl) * max_slots);
        o_segs = take(sizeof(Seg) * max_segs);
        // tile counters of a round's launches, then their staged-operand counters
        o_counters = take(sizeof(unsigned long long) * 2 * kMaxGroups);
        o_plan_state = take(sizeof(PlanState));
        o_plan_log = take(sizeof(PlanLog) * kMaxLevels);
        o_descs = take(sizeof(LevelDesc) * kPlanGroups);
        o_jobs = take(sizeof(WalkJob) * max_slots);
        o_tokens = take(sizeof(uint32_t) * kMaxTokens * max_slots);
        o_ntok = take(sizeof(int) * max_slots);
        shared_end = cur;
        LTL_CUDA_TRY(pinned_alloc(&h_probs, sizeof(Problem) * max_slots));
        LTL_CUDA_TRY(pinned_alloc(&h_ctrls, sizeof(Ctrl) * max_slots));
        LTL_CUDA_TRY(pinned_alloc(&h_staged, sizeof(unsigned long long) * kMaxGroups));
        LTL_CUDA_TRY(pinned_alloc(&h_segs, sizeof(Seg) * max_segs));
        LTL_CUDA_TRY(pinned_alloc(&h_jobs, sizeof(WalkJob) * max_slots));
        LTL_CUDA_TRY(pinned_alloc(&h_tokens, sizeof(uint32_t) * kMaxTokens * max_slots));
        LTL_CUDA_TRY(pinned_alloc(&h_ntok, sizeof(int) * max_slots));
        LTL_CUDA_TRY(pinned_alloc(&h_plan_state, sizeof(PlanState)));
        LTL_CUDA_TRY(pinned_alloc(&h_plan_log, sizeof(PlanLog) * kMaxLevels));
        LTL_CUDA_TRY(cudaEventCreate(&ev_begin));
        LTL_CUDA_TRY(cudaEventCreate(&ev_end));
        slots.resize(max_slots);
        if (opts.workspace) {
            if (((uintptr_t)opts.workspace & 255u) != 0) return fail(LTL_ERR_INVALID, "workspace must be 256-byte aligned");
            ws = (char *)opts.workspace;
            ws_bytes = opts.workspace_bytes;
            if (ws_bytes <= shared_end) return fail(LTL_ERR_OOM, "workspace too small");
            mem.reset(shared_end, ws_bytes);
        }
        return LTL_OK;
    }

    void teardown() {
        if (tuner.enabled) tuner.save();
        if (stream) cudaStreamSynchronize(stream);
        if (ws_owned && ws) {
            if (opts.free) opts.free(ws, stream, opts.user);
            else cudaFree(ws);
        }
        ws = nullptr;
        PinnedCache::get().release(h_probs);
        PinnedCache::get().release(h_ctrls);
        PinnedCache::get().release(h_staged);
        PinnedCache::get().release(h_segs);
        PinnedCache::get().release(h_jobs);
        PinnedCache::get().release(h_tokens);
        PinnedCache::get().release(h_ntok);
        PinnedCache::get().release(h_plan_state);
        PinnedCache::get().release(h_plan_log);
        PinnedCache::get().release(h_pin);
        h_pin = nullptr;
        h_probs = nullptr; h_ctrls = nullptr; h_staged = nullptr; h_segs = nullptr; h_jobs = nullptr; h_tokens = nullptr; h_ntok = nullptr;
        h_plan_state = nullptr; h_plan_log = nullptr;
        if (ev_begin) cudaEventDestroy(ev_begin);
        if (ev_end) cudaEventDestroy(ev_end);
        ev_begin = ev_end = nullptr;
        for (auto &ev : ev_op)
            if (ev) cudaEventDestroy(ev);
        ev_op.clear();
        for (auto &cg : chain_graphs) cudaGraphExecDestroy(cg.second);
        chain_graphs.clear();
        if (cap_stream) cudaStreamDestroy(cap_stream);
        cap_stream = nullptr;
        for (auto &ev : ev_chain)
            if (ev) cudaEventDestroy(ev);
        ev_chain.clear();
        for (auto &st : aux)
            if (st) {
                cudaStreamSynchronize(st);
                cudaStreamDestroy(st);
            }
        aux.clear();
        if (own_stream && stream) cudaStreamDestroy(stream);
        stream = nullptr;
        (void)cudaGetLastError();
    }

    // Without a caller workspace the engine allocates one (allocator callback
    // or cudaMalloc): `need` bytes, or 40% of the free device memory.
    ltl_status ensure_workspace(size_t need) {
        if (ws && ws_bytes >= need) return LTL_OK;
        if (opts.workspace) return fail(LTL_ERR_OOM, "workspace of %zu bytes too small (need %zu)", ws_bytes, need);
        size_t want = need;
        if (!opts.mem_budget_bytes) {
            size_t fr = 0, tot = 0;
            LTL_CUDA_TRY(cudaMemGetInfo(&fr, &tot));
            want = std::max(need, (size_t)(0.4 * (double)(fr + (ws_owned ? ws_bytes : 0))));
        }
        if (ws_owned && ws) {
            LTL_CUDA_TRY(cudaStreamSynchronize(stream));
            if (opts.free) opts.free(ws, stream, opts.user);
            else cudaFree(ws);
            ws = nullptr;
            ws_bytes = 0;
        }
        void *p = nullptr;
        if (opts.alloc) {
            p = opts.alloc(want, stream, opts.user);
            if (!p) return fail(LTL_ERR_OOM, "allocator callback returned NULL for %zu bytes", want);
        } else {
            cudaError_t e = cudaMalloc(&p, want);
            if (e != cudaSuccess) {
                (void)cudaGetLastError();
                return fail(LTL_ERR_OOM, "cudaMalloc(%zu) failed: %s", want, cudaGetErrorString(e));
            }
        }
        ws = (char *)p;
        ws_bytes = want;
        ws_owned = true;
        mem.reset(shared_end, ws_bytes);
        for (auto &s : slots) s.state = SLOT_FREE;
        return LTL_OK;
    }

    int resident() const {
        int n = 0;
        for (const auto &s : slots) n += s.state == SLOT_RUNNING;
        return n;
    }

    static const void *ws_kernel_for(const Layout &L, int op) {
        if (L.narrow) return ws_kernel_ptr_narrow(L.C, op);
        return L.Wt == 1 ? ws_kernel_ptr_w1(L.C, op) : ws_kernel_ptr_wn(L.Wt, L.C, op);
    }

    const void *kernel_for(const Layout &L, int op) const {
        if (L.ws) return ws_kernel_for(L, op);
        if (L.narrow) return fused_kernel_ptr_narrow(L.C, op);
        return L.G == 1 ? fused_kernel_ptr(L.Wt, L.C, op) : stream_kernel_ptr(L.Wt, L.C);
    }

    // Resident CTAs per SM of a kernel at a block size and dynamic shared
    // memory (opted in); cached.
    ltl_status occupancy(const void *fn, int nt, size_t smem, int &blocks) {
        if (!fn) return fail(LTL_ERR_INVALID, "no level kernel for this shape");
        LaunchCache &lc = LaunchCache::get();
        std::lock_guard<std::mutex> lk(lc.mu);
        const auto key = std::make_tuple(device, fn, nt, smem);
        const auto hit = lc.occ.find(key);
        if (hit != lc.occ.end()) {
            blocks = hit->second;
            return LTL_OK;
        }
        // the opt-in limit is an attribute of the function (the last setter
        // wins), so every level kernel is opted in once to the device maximum
        const auto fk = std::make_pair(device, fn);
        auto dyn = lc.dyn_max.find(fk);
        if (dyn == lc.dyn_max.end()) {
            int optin = 0;
            LTL_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device));
            cudaFuncAttributes fa;
            LTL_CUDA_TRY(cudaFuncGetAttributes(&fa, fn));
            const int d = optin - (int)fa.sharedSizeBytes;
            LTL_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, d));
            // all of the unified L1 / shared storage as shared memory, so that
            // shared memory does not cap the resident CTAs below the registers
            LTL_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
            dyn = lc.dyn_max.emplace(fk, d).first;
        }
        if ((long long)smem > (long long)dyn->second)
            return fail(LTL_ERR_INVALID, "problem needs %zu bytes of shared memory per CTA", smem);
        int b = 0;
        LTL_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, nt, smem));
        if (b < 1) return fail(LTL_ERR_INVALID, "level kernel cannot be resident (threads %d, smem %zu)", nt, smem);
        lc.occ.emplace(key, b);
        blocks = b;
        return LTL_OK;
    }

    // Clusters of `cl` CTAs of a cluster kernel that can be resident at once.
    ltl_status cluster_capacity(const void *fn, int nt, size_t smem, int cl, int &clusters) {
        LaunchCache &lc = LaunchCache::get();
        std::lock_guard<std::mutex> lk(lc.mu);
        const auto key = std::make_tuple(device, fn, nt, smem, cl);
        const auto hit = lc.clusters.find(key);
        if (hit != lc.clusters.end()) {
            clusters = hit->second;
            return LTL_OK;
        }
        if (cl > 8 && !lc.nonportable.count(std::make_pair(device, fn))) {
            LTL_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
            lc.nonportable.insert(std::make_pair(device, fn));
        }
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)cl;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3((unsigned)cl * (unsigned)n_sm);
        cfg.blockDim = dim3((unsigned)nt);
        cfg.dynamicSmemBytes = smem;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int n = 0;
        LTL_CUDA_TRY(cudaOccupancyMaxActiveClusters(&n, fn, &cfg));
        if (n < 1) return fail(LTL_ERR_INVALID, "no cluster of %d CTAs can be resident (smem %zu)", cl, smem);
        lc.clusters.emplace(key, n);
        clusters = n;
        return LTL_OK;
    }

    // Admits a problem into slot `si`: plans its layout for its budget (0: all
    // of the largest free block), takes its memory, uploads and packs its
    // traces.  Returns LTL_OK, or LTL_ERR_OOM when it does not fit right now.
    // `in` is moved into the slot only when the admission succeeds.
    ltl_status admit(int si, ProblemIn &in, uint64_t default_budget) {
        Slot &s = slots[si];
        Layout L;
        const uint64_t budget = in.budget ? in.budget : default_budget;
        const size_t avail = mem.largest();
        ltl_status st = plan_layout(in, opts.max_chunks, opts.level_kernel, budget, avail, L);
        if (st != LTL_OK) return st;
        size_t off = 0;
        if (!mem.alloc(L.end, off)) return fail(LTL_ERR_OOM, "no free device region of %zu bytes", L.end);
        s = Slot{};
        s.in = std::move(in);
        in = ProblemIn{};
        s.L = L;
        s.off = off;
        s.bytes = L.end;
        s.state = SLOT_RUNNING;
        s.t_admit = wall_ms();
        memset(&s.st, 0, sizeof s.st);
        char *base = ws + off;
        Ctrl *d_ctrl = (Ctrl *)(ws + o_ctrls) + si;
        const uint64_t T = L.n_traces;
        const uint32_t *d_letters = s.in.d_letters;
        const uint64_t *d_offsets = s.in.d_offsets;
        if (!s.in.device_input) {
            uint32_t *dl = (uint32_t *)(base + L.o_letters);
            uint64_t *dof = (uint64_t *)(base + L.o_offsets);
            const uint64_t np = s.in.ho[0][s.in.hn[0]], nn = s.in.ho[1][s.in.hn[1]];
            // the staged letters and offsets sit as they do in the layout
            // (offsets at the letters' size rounded up to 256 bytes), so one
            // copy moves both
            const size_t lb = round_up(4 * std::max<uint64_t>(np + nn, 1), 256),
                         need = lb + round_up(8 * (T + 1), 256);
            if (need <= kPinStageMax) {
                if (!h_pin || pin_head + need > kPinStageBytes) {
                    // every earlier staged upload has landed before the buffer is reused
                    LTL_CUDA_TRY(cudaStreamSynchronize(stream));
                    pin_head = 0;
                    if (!h_pin) LTL_CUDA_TRY(pinned_alloc(&h_pin, kPinStageBytes));
                }
                uint32_t *pl = (uint32_t *)(h_pin + pin_head);
                uint64_t *po = (uint64_t *)(h_pin + pin_head + lb);
                if (np) memcpy(pl, s.in.hl[0], 4 * np);
                if (nn) memcpy(pl + np, s.in.hl[1], 4 * nn);
                for (uint64_t i = 0; i <= s.in.hn[0]; ++i) po[i] = s.in.ho[0][i];
                for (uint64_t i = 1; i <= s.in.hn[1]; ++i) po[s.in.hn[0] + i] = np + s.in.ho[1][i];
                if ((char *)dof == (char *)dl + lb) {
                    LTL_CUDA_TRY(cudaMemcpyAsync(dl, pl, lb + 8 * (T + 1), cudaMemcpyHostToDevice, stream));
                    s.st.h2d_bytes += lb - 4 * (np + nn);   // the padding between letters and offsets
                } else {
                    if (np + nn) LTL_CUDA_TRY(cudaMemcpyAsync(dl, pl, 4 * (np + nn), cudaMemcpyHostToDevice, stream));
                    LTL_CUDA_TRY(cudaMemcpyAsync(dof, po, 8 * (T + 1), cudaMemcpyHostToDevice, stream));
                }
                pin_head += need;
            } else {
                std::vector<uint64_t> offv(T + 1);
                for (uint64_t i = 0; i <= s.in.hn[0]; ++i) offv[i] = s.in.ho[0][i];
                for (uint64_t i = 1; i <= s.in.hn[1]; ++i) offv[s.in.hn[0] + i] = np + s.in.ho[1][i];
                if (np) LTL_CUDA_TRY(cudaMemcpyAsync(dl, s.in.hl[0], 4 * np, cudaMemcpyHostToDevice, stream));
                if (nn) LTL_CUDA_TRY(cudaMemcpyAsync(dl + np, s.in.hl[1], 4 * nn, cudaMemcpyHostToDevice, stream));
                LTL_CUDA_TRY(cudaMemcpyAsync(dof, offv.data(), 8 * (T + 1), cudaMemcpyHostToDevice, stream));
                LTL_CUDA_TRY(cudaStreamSynchronize(stream));   // offv is pageable and local
            }
            s.st.h2d_bytes += 4 * (np + nn) + 8 * (T + 1);
            d_letters = dl;
            d_offsets = dof;
        }
        uint64_t *d_mask = (uint64_t *)(base + L.o_mask);
        uint64_t *d_keys = (uint64_t *)(base + L.o_keys);
        uint64_t *d_atoms = (uint64_t *)(base + L.o_atoms);
        LTL_CUDA_TRY(cudaMemsetAsync(d_ctrl, 0, sizeof(Ctrl), stream));
        // the pack launch writes every word of the mask, the atoms and the NH
        // keys, and clears the hash slots
        void *d_hslots = base + L.o_hslots;
        if (L.narrow)
            LTL_CUDA_TRY(launch_pack_narrow(d_letters, d_offsets, (uint32_t)T, L.plane, L.n_props, d_mask, d_atoms,
                                            L.stride, d_ctrl, stream, d_keys, kKeySeed, d_hslots, L.hslots));
        else
            LTL_CUDA_TRY(launch_pack(d_letters, d_offsets, (uint32_t)T, L.plane, L.W, L.Wt, L.n_props, d_mask, d_atoms,
                                     L.stride, d_ctrl, stream, d_keys, kKeySeed, d_hslots, L.hslots));
        s.st.launches += 1;
        Problem &pb = h_probs[si];
        pb = Problem{};
        pb.arena = (uint64_t *)(base + L.o_arena);
        pb.stride = L.stride;
        pb.plane = L.plane;
        pb.mask = d_mask;
        pb.keys = d_keys;
        pb.atoms = d_atoms;
        pb.prov = (uint64_t *)(base + L.o_prov);
        pb.hslots = (HSlot *)(base + L.o_hslots);
        pb.hmask = L.hslots - 1;
        pb.max_entries = L.max_entries;
        pb.ctrl = d_ctrl;
        pb.n_traces = (uint32_t)T;
        pb.n_pos = L.n_pos;
        pb.nsteps = L.nsteps;
        pb.logstep = opts.propagation == LTL_PROP_LOGSTEP ? 1u : 0u;
        pb.stop_first = opts.stop_on_solution == LTL_STOP_FIRST ? 1 : 0;
        pb.groups = L.G;
        pb.max_errors = opts.max_errors;
        // admission policy: a matrix of at most 63 bits is its own key, so the
        // hashed check of such a matrix is the exact one (Section 5)
        pb.ruc = opts.ruc;
        const uint64_t cm_bits = s.in.device_input ? T * s.in.max_len : s.in.total_pos;
        if (pb.ruc == RUC_HASH && cm_bits <= 63) pb.ruc = RUC_EXACT;
        pb.fkp_b = (uint32_t)std::max<uint64_t>(1, 63 / std::max<uint64_t>(T, 1));
        pb.key_mask = kKey63 >> std::min<uint32_t>(opts.ruc_mask_bits, 62);
        pb.spin_limit = opts.spin_limit ? opts.spin_limit : (1ull << 20);
        // uploaded with the others admitted before the next round (flush_probs)
        probs_lo = std::min(probs_lo, si);
        probs_hi = std::max(probs_hi, si);
        s.st.n_traces = T;
        s.st.words_per_trace = (uint32_t)L.W;
        s.st.threads_per_cta = (uint32_t)L.block;   // with the hash warps of the warp-specialised kernel
        s.st.traces_per_thread = (uint32_t)(L.narrow ? 4 * L.C : 2 * L.C);
        s.st.traces_per_word = L.narrow ? 2u : 1u;
        s.st.chunk_groups = L.G;
        s.st.batch = (uint32_t)L.NB;
        s.st.max_entries = L.max_entries;
        int bps = 0;
        if (occupancy(kernel_for(L, OP_U), L.block, L.G > 1 ? L.stream_smem : L.smem, bps) == LTL_OK)
            s.st.ctas_per_sm = (uint32_t)bps;
        return LTL_OK;
    }

    void release(int si) {
        Slot &s = slots[si];
        if (s.bytes) mem.release(s.off, s.bytes);
        s.bytes = 0;
        s.state = SLOT_FREE;
    }

    // Marks a slot finished with `status` (formula rebuilt later if found).
    void finish(Slot &s, ltl_status status) {
        s.state = SLOT_DONE;
        s.status = status;
        s.t_done = wall_ms();
    }

    // Closes level s.level of slot si from its control block after the level:
    // the level's counts and statistics, and whether the problem is finished
    // (invalid input, a device error, a full cache, a separator when stopping
    // at one, or max_size reached).
    void close_level(int si, const Ctrl &h, std::vector<int> &found_slots) {
        Slot &s = slots[si];
        const int k = s.level;
        if (h.invalid_letter) {
            s.error = "trace letters use propositions >= n_props, offsets decrease, or a trace exceeds max_len";
            finish(s, LTL_ERR_INVALID);
            return;
        }
        if (h.err) {
            s.error = h.err == LTL_ERR_INVALID ? "launch shape / shared memory mismatch"
                                               : "device wait exceeded spin_limit";
            finish(s, (ltl_status)h.err);
            return;
        }
        const uint64_t ent = std::min<uint64_t>(h.n_entries, s.L.max_entries);
        s.lvl_count[k] = ent - s.prev_entries;
        s.st.unique[k] = ent - s.prev_entries;
        s.st.candidates[k] = h.cands - s.prev_cands;
        s.prev_entries = ent;
        s.prev_cands = h.cands;
        s.st.entries = ent;
        s.st.compares = h.compares;
        s.st.collisions = h.collisions;
        const bool stopped_early = (h.stop != 0) || h.cap_hit;
        if (!stopped_early) s.st.levels_done = k;
        if (h.found_count > 0) s.found = true;
        if (h.cap_hit) {
            if (s.found) found_slots.push_back(si);
            finish(s, s.found ? LTL_OK : LTL_CAP_REACHED);
            return;
        }
        if (s.found && opts.stop_on_solution != LTL_STOP_NONE) {
            found_slots.push_back(si);
            finish(s, LTL_OK);
            return;
        }
        if (++s.level > s.in.max_size) {
            if (s.found) found_slots.push_back(si);
            finish(s, s.found ? LTL_OK : LTL_NOT_FOUND);
        }
    }

    // A level without candidates (no connective fits its cost): nothing runs.
    void close_empty_level(int si, std::vector<int> &found_slots) {
        Slot &s = slots[si];
        s.lvl_count[s.level] = 0;
        s.st.levels_done = s.level;
        if (++s.level > s.in.max_size) {
            if (s.found) found_slots.push_back(si);
            finish(s, s.found ? LTL_OK : LTL_NOT_FOUND);
        }
    }

    // Levels s.level, s.level + 1, ... that the device may plan: each stays
    // below kConcurrentBelow candidates even if every candidate of the levels
    // before it were new (exact for the first, whose operand counts are
    // known; an upper bound after it).  Per level, the connectives that can
    // have candidates (under those bounds) and their candidate bounds.
    struct ChainLevel {
        uint64_t cands[8];
        bool has[8];
    };
    int chain_length(const Slot &s, const Costs &cost, std::vector<ChainLevel> &lv) const {
        uint64_t beg[kMaxLevels] = {}, cnt[kMaxLevels] = {};
        for (int j = 1; j < s.level && j < kMaxLevels; ++j) cnt[j] = s.lvl_count[j];
        lv.clear();
        for (int j = s.level; j <= s.in.max_size && j < kMaxLevels; ++j) {
            ChainLevel c{};
            uint64_t total = 0;
            auto emit = [&](Seg sg) {
                const uint64_t n = seg_candidates(sg);
                c.cands[sg.op] += n;
                c.has[sg.op] = true;
                total += n;
            };
            plan_level_segments(s.in.ops, s.in.n_props, beg, cnt, j, cost, emit);
            if (total >= kConcurrentBelow) break;
            cnt[j] = total;
            lv.push_back(c);
        }
        return (int)lv.size();
    }

    // The instantiated graph of a chain with this key.  Capturing and
    // instantiating costs about as much as a few direct enqueues save, so a
    // shape is enqueued directly (null) until it has been seen
    // kChainCaptureAfter times; then `enqueue` is captured on a capture
    // stream and instantiated (null when capture is not possible).
    template <class Enqueue>
    cudaGraphExec_t chain_graph(const std::string &key, Enqueue &enqueue) {
        auto hit = chain_graphs.find(key);
        if (hit != chain_graphs.end()) return hit->second;
        if (++chain_seen[key] < kChainCaptureAfter) {
            if (chain_seen.size() > kChainShapes) chain_seen.clear();
            return nullptr;
        }
        chain_seen.erase(key);
        if (!cap_stream && cudaStreamCreateWithFlags(&cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
            (void)cudaGetLastError();
            cap_stream = nullptr;
            return nullptr;
        }
        cudaGraph_t g = nullptr;
        cudaGraphExec_t exec = nullptr;
        if (cudaStreamBeginCapture(cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            (void)cudaGetLastError();
            return nullptr;
        }
        const cudaError_t e = enqueue(cap_stream);
        const cudaError_t ee = cudaStreamEndCapture(cap_stream, &g);
        if (e != cudaSuccess || ee != cudaSuccess || !g || cudaGraphInstantiate(&exec, g, 0) != cudaSuccess) {
            (void)cudaGetLastError();
            if (g) cudaGraphDestroy(g);
            return nullptr;
        }
        cudaGraphDestroy(g);
        if (chain_graphs.size() >= kChainShapes) {
            cudaGraphExecDestroy(chain_graphs.begin()->second);
            chain_graphs.erase(chain_graphs.begin());
        }
        chain_graphs.emplace(key, exec);
        return exec;
    }

    // Runs the levels of `lv` for slot si planned on the device: per level the
    // planner kernel (closing the level before), then one launch per
    // connective with its extent in device memory -- concurrent on the
    // auxiliary streams -- and after the last level one more planner call
    // that closes it.  One read-back of the level logs, then each level is
    // closed on the host exactly as a host-planned level would be.
    ltl_status run_chain(int si, const Costs &cost, const std::vector<ChainLevel> &lv) {
        Slot &s = slots[si];
        const Layout &L = s.L;
        const int k0 = s.level, m = (int)lv.size();
        memset(h_plan_state, 0, sizeof(PlanState));
        for (int j = 1; j < k0; ++j) {
            h_plan_state->lvl_begin[j] = s.lvl_begin[j];
            h_plan_state->lvl_count[j] = s.lvl_count[j];
        }
        PlanState *d_state = (PlanState *)(ws + o_plan_state);
        PlanLog *d_log = (PlanLog *)(ws + o_plan_log);
        LevelDesc *d_desc = (LevelDesc *)(ws + o_descs);
        Seg *d_segs = (Seg *)(ws + o_segs);
        unsigned long long *d_counters = (unsigned long long *)(ws + o_counters);
        while ((int)aux.size() < kAuxStreams) {
            cudaStream_t st = nullptr;
            LTL_CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
            aux.push_back(st);
        }
        PlanArgs pa{};
        pa.prob = (const Problem *)(ws + o_probs) + si;
        pa.state = d_state;
        pa.log = d_log;
        pa.segs = d_segs;
        pa.desc = d_desc;
        pa.counters = d_counters;
        pa.cost = cost;
        pa.ops = s.in.ops;
        pa.n_props = s.in.n_props;
        pa.stop_mode = opts.stop_on_solution;
        pa.prob_index = si;
        pa.nb = L.NB;
        pa.tiles_per_cta = tune_choice(kTuneDefault).tiles_per_cta;
        // fork / join events of the concurrent launches: level start, then one per launch
        const int per_level = 1 + kPlanGroups;
        while ((int)ev_chain.size() < m * per_level) {
            cudaEvent_t ev = nullptr;
            LTL_CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
            ev_chain.push_back(ev);
        }
        // per level: the planner's arguments and the launches (connective, kernel, CTAs)
        struct LevelLaunches {
            PlanArgs pa;
            std::vector<const void *> fns;
            std::vector<int> grids;
        };
        std::vector<LevelLaunches> plan(m);
        std::vector<std::vector<int>> level_ops(m);
        const int order[8] = {OP_ATOM, OP_F, OP_U, OP_G, OP_X, OP_AND, OP_OR, OP_NOT};
        std::string key((const char *)&ws, sizeof ws);   // what the enqueued work depends on
        auto add_key = [&key](const void *p, size_t n) { key.append((const char *)p, n); };
        add_key(&si, sizeof si);
        add_key(&k0, sizeof k0);
        add_key(&L.block, sizeof L.block);
        add_key(&L.smem, sizeof L.smem);
        for (int i = 0; i < m; ++i) {
            LevelLaunches &ll = plan[i];
            ll.pa = pa;
            ll.pa.n_groups = 0;
            for (int op : order) {
                if (!lv[i].has[op]) continue;
                const void *fn = kernel_for(L, op);
                int bps = 0;
                ltl_status st = occupancy(fn, L.block, L.smem, bps);
                if (st != LTL_OK) return st;
                const uint64_t cap = (uint64_t)bps * (uint64_t)n_sm;
                const uint64_t want = std::max<uint64_t>(1, (lv[i].cands[op] + L.NB - 1) / L.NB);
                const int grid = (int)std::min<uint64_t>(cap, want);
                ll.pa.group_op[ll.pa.n_groups] = op;
                ll.pa.group_cap[ll.pa.n_groups] = (uint32_t)grid;
                ll.pa.n_groups++;
                ll.fns.push_back(fn);
                ll.grids.push_back(grid);
                level_ops[i].push_back(op);
            }
            add_key(&ll.pa, sizeof ll.pa);
            add_key(ll.fns.data(), sizeof(const void *) * ll.fns.size());
            add_key(ll.grids.data(), sizeof(int) * ll.grids.size());
        }
        // the whole chain, enqueued on st0 (forking onto the auxiliary streams)
        auto enqueue = [&](cudaStream_t st0) -> cudaError_t {
            cudaError_t e = cudaMemcpyAsync(d_state, h_plan_state, sizeof(PlanState), cudaMemcpyHostToDevice, st0);
            for (int i = 0; i < m && e == cudaSuccess; ++i) {
                const LevelLaunches &ll = plan[i];
                e = launch_plan(ll.pa, k0 + i, i > 0, true, st0);
                cudaEvent_t ev_lb = ev_chain[i * per_level];
                if (e == cudaSuccess) e = cudaEventRecord(ev_lb, st0);
                const bool concurrent = ll.pa.n_groups > 1;
                for (int g = 0; g < ll.pa.n_groups && e == cudaSuccess; ++g) {
                    LevelArgs la{};
                    la.segs = d_segs + (size_t)g * kPlanSegsPerGroup;
                    la.probs = (const Problem *)(ws + o_probs);
                    la.tile_counter = d_counters + g;
                    la.desc = d_desc + g;
                    void *args[] = {&la};
                    cudaStream_t st = st0;
                    if (concurrent) {
                        st = aux[g % aux.size()];
                        e = cudaStreamWaitEvent(st, ev_lb, 0);
                    }
                    if (e == cudaSuccess) e = cudaLaunchKernel(ll.fns[g], dim3(ll.grids[g]), dim3(L.block), args, L.smem, st);
                    if (e == cudaSuccess) e = cudaEventRecord(ev_chain[i * per_level + 1 + g], st);
                }
                if (concurrent)
                    for (int g = 0; g < ll.pa.n_groups && e == cudaSuccess; ++g)
                        e = cudaStreamWaitEvent(st0, ev_chain[i * per_level + 1 + g], 0);
            }
            if (e == cudaSuccess) {
                PlanArgs last = pa;
                last.n_groups = 0;
                e = launch_plan(last, k0 + m, true, false, st0);
            }
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(h_plan_log + k0, d_log + k0, sizeof(PlanLog) * m, cudaMemcpyDeviceToHost, st0);
            return e;
        };
        // a chain of the same shape runs as one CUDA graph, captured once
        cudaGraphExec_t exec = chain_graph(key, enqueue);
        if (exec) {
            LTL_CUDA_TRY(cudaGraphLaunch(exec, stream));
        } else {
            LTL_CUDA_TRY(enqueue(stream));
        }
        LTL_CUDA_TRY(cudaStreamSynchronize(stream));
        total_rounds += (uint64_t)m;
        std::vector<int> found_slots;
        for (int i = 0; i < m && s.state == SLOT_RUNNING; ++i) {
            const int k = k0 + i;
            const PlanLog &lg = h_plan_log[k];
            if (!lg.ran) break;   // the device stopped the chain (the host closes the same way)
            s.st.device_planned_levels++;
            if (exec) s.st.graph_levels++;
            s.st.launches += 1 + (uint32_t)level_ops[i].size();   // planner + launches
            s.st.d2h_bytes += sizeof(PlanLog);
            s.lvl_begin[k] = lg.begin;
            if (lg.n_segs == 0) {
                close_empty_level(si, found_slots);
                continue;
            }
            // device clock from this level's planner call to the next one
            const float level_ms = lg.t_end > lg.t_begin ? (float)((double)(lg.t_end - lg.t_begin) * 1e-6) : 0.f;
            for (int op : level_ops[i]) {
                s.st.op_ms[k][op] = level_ms;
                s.st.op_kernel[k][op] = LTL_LAUNCH_FUSED;   // chains run the fused kernel
            }
            s.rounds++;
            s.st.ms[k] = level_ms;
            h_ctrls[si] = lg.snap;
            close_level(si, lg.snap, found_slots);
        }
        s.st.launches += 1;   // the closing planner call
        return rebuild_formulas(found_slots);
    }

    // One round: the next size level of every running problem.
    // The descriptors of the problems admitted since the last round, in one
    // copy of the slot range they span (the slots between hold the
    // descriptors of running or free slots, unchanged).
    ltl_status flush_probs() {
        if (probs_hi < probs_lo) return LTL_OK;
        LTL_CUDA_TRY(cudaMemcpyAsync((Problem *)(ws + o_probs) + probs_lo, &h_probs[probs_lo],
                                     sizeof(Problem) * (size_t)(probs_hi - probs_lo + 1), cudaMemcpyHostToDevice,
                                     stream));
        probs_lo = INT32_MAX;
        probs_hi = -1;
        return LTL_OK;
    }

    ltl_status round() {
        {
            const ltl_status fs = flush_probs();
            if (fs != LTL_OK) return fs;
        }
        Costs cost;
        // 0 reads as 1; anything above the largest level only bans the connective
        for (int i = 0; i < 8; ++i)
            cost.c[i] = opts.costs[i] ? (int)std::min<uint32_t>(opts.costs[i], kMaxLevels) : 1;
        // one problem on the fused kernel: its small levels are planned on the device
        if (opts.level_planning == LTL_PLAN_AUTO && max_slots == 1 && slots[0].state == SLOT_RUNNING &&
            !slots[0].L.ws && slots[0].L.G == 1) {
            std::vector<ChainLevel> lv;
            if (chain_length(slots[0], cost, lv) >= 2) return run_chain(0, cost, lv);
        }
        std::vector<Seg> segs;
        std::vector<int> ran;   // slots that enumerate a level this round
        std::vector<int> found_slots;
        for (int si = 0; si < max_slots; ++si) {
            Slot &s = slots[si];
            while (s.state == SLOT_RUNNING) {
                const int k = s.level;
                s.lvl_begin[k] = s.prev_entries;
                const size_t before = segs.size();
                level_segments(s, k, si, cost, segs);
                if (segs.size() > before) {
                    ran.push_back(si);
                    break;
                }
                close_empty_level(si, found_slots);
            }
        }
        if (ran.empty()) return rebuild_formulas(found_slots);
        if (segs.size() > max_segs) return fail(LTL_ERR_INVALID, "too many segments in one round");
        // group by launch (kernel, block size); a group's shared memory is the
        // largest any of its problems needs
        struct Group {
            const void *fn;
            int nt, op, nb;
            size_t smem;
            std::vector<int> seg_ids;
            int cl = 0;        // cluster size of the cluster kernel
            bool ws = false;   // the warp-specialised kernel
            int kind = 0;      // LTL_LAUNCH_*
        };
        std::vector<Group> groups;
        // Matrices larger than one CTA: the cluster kernel (one candidate over
        // a cluster's SMs) for a problem whose round has fewer candidates than
        // there are SMs -- the streaming kernel would leave SMs idle -- and
        // the two-pass streaming kernel otherwise (measured faster per SM when
        // every SM has candidates of its own).
        std::vector<uint64_t> prob_cands(max_slots, 0);
        for (const Seg &sg : segs) prob_cands[sg.prob] += seg_candidates(sg);
        // Matrices that fit one CTA: the warp-specialised kernel (hash warps
        // settle batches while the compute warps go on) for a problem whose
        // round has at least kWsAutoMin candidates, the fused kernel for the
        // smaller rounds, which are bound by launch and drain latency.
        for (int i = 0; i < (int)segs.size(); ++i) {
            const Slot &s = slots[segs[i].prob];
            const bool cluster =
                s.L.CL > 0 && (opts.level_kernel == LTL_KERNEL_WS || prob_cands[segs[i].prob] < (uint64_t)n_sm);
            const bool auto_ws = !cluster && !s.L.ws && s.L.ws_ok && opts.level_kernel == LTL_KERNEL_AUTO &&
                                 prob_cands[segs[i].prob] >= kWsAutoMin;
            const void *fn = cluster   ? cluster_kernel_ptr(s.L.Wt, s.L.C)
                             : auto_ws ? ws_kernel_for(s.L, segs[i].op)
                                       : kernel_for(s.L, segs[i].op);
            const int cl = cluster ? s.L.CL : 0;
            const int nt = auto_ws ? s.L.NT + kWsExtraThreads : s.L.block;
            const size_t smem = cluster        ? s.L.smem
                                : s.L.G > 1    ? s.L.stream_smem
                                : auto_ws      ? s.L.ws_smem
                                               : s.L.smem;
            int g = -1;
            for (int j = 0; j < (int)groups.size(); ++j)
                if (groups[j].fn == fn && groups[j].nt == nt && groups[j].cl == cl) g = j;
            if (g < 0) {
                const int kind = cluster                 ? LTL_LAUNCH_CLUSTER
                                 : (auto_ws || s.L.ws)   ? LTL_LAUNCH_WS
                                 : s.L.G > 1             ? LTL_LAUNCH_STREAM
                                                         : LTL_LAUNCH_FUSED;
                groups.push_back(Group{fn, nt, segs[i].op, s.L.NB, 0, {}, cl, auto_ws || s.L.ws, kind});
                g = (int)groups.size() - 1;
            }
            groups[g].smem = std::max(groups[g].smem, smem);
            groups[g].seg_ids.push_back(i);
        }
        if ((int)groups.size() > kMaxGroups) return fail(LTL_ERR_INVALID, "too many launches in one round");
        // tiles: about four per resident CTA in every launch
        size_t n_out = 0;
        std::vector<size_t> first(groups.size());
        std::vector<uint64_t> tiles(groups.size());
        std::vector<int> grid(groups.size());
        std::vector<uint64_t> gcands(groups.size(), 0);
        uint64_t round_cands = 0;
        for (size_t g = 0; g < groups.size(); ++g) {
            for (int i : groups[g].seg_ids) gcands[g] += seg_candidates(segs[i]);
            round_cands += gcands[g];
        }
        // launches run concurrently in small rounds (bound by launch latency)
        // and whenever the round holds several problems (batches, servers:
        // many launch shapes, each launch small); a large round of one problem
        // keeps its launches in order, so that each has an event time of its own
        const bool concurrent = groups.size() > 1 && (round_cands < kRoundConcurrentBelow || ran.size() > 1);
        // a larger round of one problem: its U launch, the level's longest, runs
        // alone first, timed by its own events; the other launches follow it
        // concurrently (in order their tails add up)
        int lead = -1;
        if (!concurrent && groups.size() > 2)
            for (size_t g = 0; g < groups.size(); ++g)
                if (groups[g].op == OP_U && (lead < 0 || gcands[g] > gcands[lead])) lead = (int)g;
        const bool split = lead >= 0;
        std::vector<int> choice(groups.size(), -1);
        std::vector<std::string> tkey(groups.size());
        for (size_t g = 0; g < groups.size(); ++g) {
            Group &gr = groups[g];
            int bps = 0;
            ltl_status st = occupancy(gr.fn, gr.nt, gr.smem, bps);
            if (st != LTL_OK) return st;
            const uint64_t cands = gcands[g];
            int c = kTuneDefault;
            // launches that run alone are tuned (their event times are their own)
            if (tuner.enabled && !concurrent && (!split || (int)g == lead) && cands >= kTuneMinCands) {
                const Slot &s0 = slots[segs[gr.seg_ids[0]].prob];
                char key[96];
                snprintf(key, sizeof key, "%s%dc%dt%d%s-op%d-b%d", s0.L.narrow ? "n" : "w", s0.L.Wt, s0.L.C, gr.nt,
                         gr.ws ? "ws" : (s0.L.G > 1 ? "st" : "fu"), gr.op, ceil_log2(cands));
                tkey[g] = key;
                c = choice[g] = tuner.pick(tkey[g], bps > 1 && !gr.cl);
            }
            const TuneChoice tc = tune_choice(c);
            // persistent workers: CTAs, or clusters for the cluster kernel
            uint64_t cap = (uint64_t)std::max(1, bps - tc.cta_less) * (uint64_t)n_sm;
            if (gr.cl) {
                int nclusters = 0;
                st = cluster_capacity(gr.fn, gr.nt, gr.smem, gr.cl, nclusters);
                if (st != LTL_OK) return st;
                cap = (uint64_t)nclusters;
            }
            const uint32_t cpt = tile_target(cands, cap, gr.nb, tc.tiles_per_cta);
            uint64_t total = 0;
            first[g] = n_out;
            for (int i : gr.seg_ids) {
                Seg sg = segs[i];
                set_tiles(sg, cpt);
                sg.tile_begin = total;
                total += sg.n_tiles;
                h_segs[n_out++] = sg;
            }
            tiles[g] = total;
            grid[g] = (int)std::min<uint64_t>(total, cap);
        }
        while (ev_op.size() < groups.size()) {
            cudaEvent_t ev = nullptr;
            LTL_CUDA_TRY(cudaEventCreate(&ev));
            ev_op.push_back(ev);
        }
        Seg *d_segs = (Seg *)(ws + o_segs);
        unsigned long long *d_counters = (unsigned long long *)(ws + o_counters);
        LTL_CUDA_TRY(cudaMemcpyAsync(d_segs, h_segs, sizeof(Seg) * n_out, cudaMemcpyHostToDevice, stream));
        LTL_CUDA_TRY(cudaMemsetAsync(d_counters, 0, sizeof(unsigned long long) * 2 * kMaxGroups, stream));
        LTL_CUDA_TRY(cudaEventRecord(ev_begin, stream));
        if (concurrent || split)
            while ((int)aux.size() < kAuxStreams) {
                cudaStream_t st = nullptr;
                LTL_CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
                aux.push_back(st);
            }
        // launch order: the lead launch first when the round is split
        std::vector<size_t> order;
        if (split) order.push_back((size_t)lead);
        for (size_t g = 0; g < groups.size(); ++g)
            if ((int)g != lead) order.push_back(g);
        for (size_t oi = 0; oi < order.size(); ++oi) {
            const size_t g = order[oi];
            LevelArgs la{};
            la.segs = d_segs + first[g];
            la.probs = (const Problem *)(ws + o_probs);
            la.tile_counter = d_counters + g;
            la.staged = d_counters + kMaxGroups + g;
            la.n_segs = (int)groups[g].seg_ids.size();
            la.total_tiles = tiles[g];
            void *args[] = {&la};
            cudaStream_t st = stream;
            if (concurrent) {
                st = aux[g % aux.size()];
                LTL_CUDA_TRY(cudaStreamWaitEvent(st, ev_begin, 0));
            } else if (split && (int)g != lead) {
                st = aux[oi % aux.size()];
                LTL_CUDA_TRY(cudaStreamWaitEvent(st, ev_op[lead], 0));
            }
            if (grid[g] > 0 && groups[g].cl) {
                // grid[g] clusters of cl CTAs
                cudaLaunchConfig_t cfg = {};
                cudaLaunchAttribute attr[1];
                attr[0].id = cudaLaunchAttributeClusterDimension;
                attr[0].val.clusterDim.x = (unsigned)groups[g].cl;
                attr[0].val.clusterDim.y = 1;
                attr[0].val.clusterDim.z = 1;
                cfg.gridDim = dim3((unsigned)grid[g] * (unsigned)groups[g].cl);
                cfg.blockDim = dim3((unsigned)groups[g].nt);
                cfg.dynamicSmemBytes = groups[g].smem;
                cfg.stream = st;
                cfg.attrs = attr;
                cfg.numAttrs = 1;
                LTL_CUDA_TRY(cudaLaunchKernelExC(&cfg, groups[g].fn, args));
            } else if (grid[g] > 0) {
                LTL_CUDA_TRY(cudaLaunchKernel(groups[g].fn, dim3(grid[g]), dim3(groups[g].nt), args, groups[g].smem, st));
            }
            LTL_CUDA_TRY(cudaEventRecord(ev_op[g], st));
        }
        if (concurrent || split)
            for (size_t g = 0; g < groups.size(); ++g)
                if ((int)g != lead) LTL_CUDA_TRY(cudaStreamWaitEvent(stream, ev_op[g], 0));
        int hi = 0;
        for (int si : ran) hi = std::max(hi, si + 1);
        LTL_CUDA_TRY(cudaMemcpyAsync(h_ctrls, ws + o_ctrls, sizeof(Ctrl) * hi, cudaMemcpyDeviceToHost, stream));
        LTL_CUDA_TRY(cudaMemcpyAsync(h_staged, d_counters + kMaxGroups, sizeof(unsigned long long) * groups.size(),
                                     cudaMemcpyDeviceToHost, stream));
        LTL_CUDA_TRY(cudaStreamSynchronize(stream));
        ++total_rounds;
        // per launch: its own time when launches ran one after another (the
        // lead launch of a split round included); from the start of the round
        // when they ran concurrently; from the end of the lead launch for the
        // others of a split round
        float round_ms = 0.f;
        std::vector<float> op_ms(groups.size());
        for (size_t g = 0; g < groups.size(); ++g) {
            float t = 0.f;
            cudaEvent_t from = ev_begin;
            if (split) from = (int)g == lead ? ev_begin : ev_op[lead];
            else if (!concurrent && g > 0) from = ev_op[g - 1];
            LTL_CUDA_TRY(cudaEventElapsedTime(&t, from, ev_op[g]));
            op_ms[g] = t;
            if (choice[g] >= 0) tuner.record(tkey[g], choice[g], 1e6 * (double)t / (double)gcands[g]);
            float since = 0.f;
            LTL_CUDA_TRY(cudaEventElapsedTime(&since, ev_begin, ev_op[g]));
            round_ms = std::max(round_ms, since);
        }
        // per problem and launch (a problem's segments of one connective are
        // in one launch): the launch's time, kernel and staged operands, and
        // the launch counted once for each problem it served -- one pass over
        // the segments, before the levels are closed
        std::vector<int> stamp(max_slots, -1);
        for (size_t g = 0; g < groups.size(); ++g)
            for (int i : groups[g].seg_ids) {
                const int p = segs[i].prob;
                if (stamp[p] == (int)g) continue;
                stamp[p] = (int)g;
                Slot &s = slots[p];
                const int k = s.level, op = groups[g].op;
                s.st.op_ms[k][op] = op_ms[g];
                s.st.op_kernel[k][op] = (uint8_t)groups[g].kind;
                s.st.op_alone[k][op] = (!concurrent && (!split || (int)g == lead)) ? 1 : 0;
                s.st.op_staged[k][op] = h_staged[g];
                s.st.launches += 1;
            }
        // close the level of every problem that ran
        for (int si : ran) {
            Slot &s = slots[si];
            const Ctrl &h = h_ctrls[si];
            s.rounds++;
            s.st.ms[s.level] = round_ms;
            s.st.d2h_bytes += sizeof(Ctrl) + sizeof(unsigned long long) * groups.size();
            close_level(si, h, found_slots);
        }
        return rebuild_formulas(found_slots);
    }

    // One provenance walk for every problem that found a separator.
    ltl_status rebuild_formulas(const std::vector<int> &found_slots) {
        if (found_slots.empty()) return LTL_OK;
        const int n = (int)found_slots.size();
        for (int j = 0; j < n; ++j) {
            const int si = found_slots[j];
            const Slot &s = slots[si];
            h_jobs[j].prov = (const uint64_t *)(ws + s.off + s.L.o_prov);
            h_jobs[j].n_entries = s.prev_entries;
            h_jobs[j].root = h_ctrls[si].found_prov;
        }
        WalkJob *d_jobs = (WalkJob *)(ws + o_jobs);
        uint32_t *d_tokens = (uint32_t *)(ws + o_tokens);
        int *d_ntok = (int *)(ws + o_ntok);
        LTL_CUDA_TRY(cudaMemcpyAsync(d_jobs, h_jobs, sizeof(WalkJob) * n, cudaMemcpyHostToDevice, stream));
        LTL_CUDA_TRY(launch_walk_batch(d_jobs, n, d_tokens, kMaxTokens, d_ntok, stream));
        LTL_CUDA_TRY(cudaMemcpyAsync(h_tokens, d_tokens, sizeof(uint32_t) * kMaxTokens * n, cudaMemcpyDeviceToHost,
                                     stream));
        LTL_CUDA_TRY(cudaMemcpyAsync(h_ntok, d_ntok, sizeof(int) * n, cudaMemcpyDeviceToHost, stream));
        LTL_CUDA_TRY(cudaStreamSynchronize(stream));
        for (int j = 0; j < n; ++j) {
            Slot &s = slots[found_slots[j]];
            s.st.launches += 1;
            s.st.d2h_bytes += sizeof(uint32_t) * kMaxTokens + sizeof(int);
            if (h_ntok[j] <= 0) {
                s.status = LTL_ERR_CUDA;
                s.error = "provenance walk failed";
                continue;
            }
            s.formula.clear();
            tokens_to_text(h_tokens + (size_t)j * kMaxTokens, h_ntok[j], 0, s.formula);
            s.st.found_size = h_ctrls[found_slots[j]].found_level;
        }
        return LTL_OK;
    }

    // Formula text of cache entry idx of slot si (for introspection).
    ltl_status entry_formula(int si, uint64_t idx, std::string &text) {
        const Slot &s = slots[si];
        uint64_t p = 0;
        LTL_CUDA_TRY(cudaMemcpyAsync(&h_jobs[0].root, ws + s.off + s.L.o_prov + 8 * idx, 8, cudaMemcpyDeviceToHost,
                                     stream));
        LTL_CUDA_TRY(cudaStreamSynchronize(stream));
        p = h_jobs[0].root;
        h_jobs[0].prov = (const uint64_t *)(ws + s.off + s.L.o_prov);
        h_jobs[0].n_entries = s.prev_entries;
        h_jobs[0].root = p;
        WalkJob *d_jobs = (WalkJob *)(ws + o_jobs);
        LTL_CUDA_TRY(cudaMemcpyAsync(d_jobs, h_jobs, sizeof(WalkJob), cudaMemcpyHostToDevice, stream));
        LTL_CUDA_TRY(launch_walk_batch(d_jobs, 1, (uint32_t *)(ws + o_tokens), kMaxTokens, (int *)(ws + o_ntok), stream));
        LTL_CUDA_TRY(cudaMemcpyAsync(h_tokens, ws + o_tokens, sizeof(uint32_t) * kMaxTokens, cudaMemcpyDeviceToHost,
                                     stream));
        LTL_CUDA_TRY(cudaMemcpyAsync(h_ntok, ws + o_ntok, sizeof(int), cudaMemcpyDeviceToHost, stream));
        LTL_CUDA_TRY(cudaStreamSynchronize(stream));
        if (h_ntok[0] <= 0) return fail(LTL_ERR_CUDA, "provenance walk failed");
        text.clear();
        tokens_to_text(h_tokens, h_ntok[0], 0, text);
        return LTL_OK;
    }

    void fill_result(const Slot &s, ltl_result &r) const {
        memset(&r, 0, sizeof r);
        r.id = s.in.id;
        r.status = s.status;
        r.found_size = s.status == LTL_OK ? s.st.found_size : 0;
        r.levels_done = s.st.levels_done;
        snprintf(r.formula, sizeof r.formula, "%s", s.status == LTL_OK ? s.formula.c_str() : "");
        for (int k = 0; k < kMaxLevels; ++k) {
            r.unique[k] = s.st.unique[k];
            r.candidates[k] = s.st.candidates[k];
        }
        r.n_traces = s.st.n_traces;
        r.rounds = s.rounds;
        r.queue_ms = s.t_admit - s.in.t_submit;
        r.latency_ms = s.t_done - s.in.t_submit;
    }
};

// Host threads for large copies, started once per process: run(k, fn) calls
// fn(0..k-1), one part on the calling thread and the others on the pool, and
// returns when all are done.  Callers of run() take turns.  The pool is never
// torn down (its idle threads wait on a condition variable; at process exit
// they are simply ended), so no exit path waits on it.
class CopyPool {
public:
    static CopyPool &get() {
        static CopyPool *p = new CopyPool();
        return *p;
    }
    int workers() const { return (int)n_workers; }
    template <class F>
    void run(int k, const F &fn) {
        std::lock_guard<std::mutex> turn(run_mu);
        std::function<void(int)> f(fn);
        {
            std::lock_guard<std::mutex> lk(mu);
            job = &f;
            n_parts = k;
            next = 1;   // part 0 is the caller's
            left = k;
            ++gen;
        }
        cv.notify_all();
        f(0);
        take_parts();
        std::unique_lock<std::mutex> lk(mu);
        if (--left > 0) cv_done.wait(lk, [&] { return left == 0; });
        job = nullptr;
    }

private:
    CopyPool() {
        const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
        n_workers = std::min(7u, hw > 1 ? hw - 1 : 0u);
        for (unsigned i = 0; i < n_workers; ++i) std::thread([this] { loop(); }).detach();
    }
    // parts not yet started, taken by whichever thread is free
    void take_parts() {
        for (;;) {
            int i;
            const std::function<void(int)> *f;
            {
                std::lock_guard<std::mutex> lk(mu);
                if (!job || next >= n_parts) return;
                i = next++;
                f = job;
            }
            (*f)(i);
            std::lock_guard<std::mutex> lk(mu);
            if (--left == 0) cv_done.notify_all();
        }
    }
    void loop() {
        uint64_t seen = 0;
        for (;;) {
            {
                std::unique_lock<std::mutex> lk(mu);
                cv.wait(lk, [&] { return gen != seen; });
                seen = gen;
            }
            take_parts();
        }
    }
    unsigned n_workers = 0;
    std::mutex run_mu, mu;
    std::condition_variable cv, cv_done;
    const std::function<void(int)> *job = nullptr;
    int n_parts = 0, next = 0, left = 0;
    uint64_t gen = 0;
};

// A host copy of n elements (at least one, zero when n is 0).  Large inputs
// are copied in parts on the copy pool, each part's thread also
// first-touching its share of the fresh, uninitialised allocation: one thread
// copying a request of 15 MB took about 1 ms, most of it page faults.
template <class T>
std::unique_ptr<T[]> copy_parallel(const T *src, uint64_t n) {
    std::unique_ptr<T[]> dst(new (std::nothrow) T[n ? n : 1]);
    if (!dst) return dst;   // out of host memory: the caller reports it
    if (n == 0) {
        dst[0] = T();
        return dst;
    }
    const uint64_t bytes = n * sizeof(T);
    CopyPool &pool = CopyPool::get();
    const uint64_t k = std::min<uint64_t>((uint64_t)pool.workers() + 1, std::max<uint64_t>(1, bytes >> 21));
    if (k <= 1) {
        memcpy(dst.get(), src, bytes);
        return dst;
    }
    const uint64_t per = (n + k - 1) / k;
    T *d = dst.get();
    pool.run((int)k, [d, src, n, per](int i) {
        const uint64_t b = (uint64_t)i * per, e = std::min(n, b + per);
        if (b < e) memcpy(d + b, src + b, (e - b) * sizeof(T));
    });
    return dst;
}

// Builds the ProblemIn of host traces (copying them when `own`).
ltl_status problem_from_host(const ltl_traces *P, const ltl_traces *N, int n_props, uint32_t ops, int max_size,
                             uint64_t budget, bool own, ProblemIn &in) {
    ltl_status s = check_common(n_props, ops, max_size);
    if (s != LTL_OK) return s;
    if ((s = check_traces(P, "P")) != LTL_OK) return s;
    if ((s = check_traces(N, "N")) != LTL_OK) return s;
    // a request's latency counts from here, the library's copy of its traces included
    in.t_submit = wall_ms();
    const ltl_traces *tr[2] = {P, N};
    for (int h = 0; h < 2; ++h) {
        in.hn[h] = tr[h]->n_traces;
        if (own) {
            const uint64_t np = tr[h]->offsets[tr[h]->n_traces];
            in.own_l[h] = copy_parallel(tr[h]->letters, np);
            in.own_o[h] = copy_parallel(tr[h]->offsets, tr[h]->n_traces + 1);
            if (!in.own_l[h] || !in.own_o[h]) return fail(LTL_ERR_OOM, "no host memory for a copy of the traces");
            in.hl[h] = in.own_l[h].get();
            in.ho[h] = in.own_o[h].get();
        } else {
            in.hl[h] = tr[h]->letters;
            in.ho[h] = tr[h]->offsets;
        }
    }
    in.n_pos = P->n_traces;
    in.n_neg = N->n_traces;
    in.max_len = std::max(traces_max_len(P), traces_max_len(N));
    in.total_pos = P->offsets[P->n_traces] + N->offsets[N->n_traces];
    in.n_props = n_props;
    in.ops = ops;
    in.max_size = max_size;
    in.budget = budget;
    return LTL_OK;
}

ltl_opts default_opts() {
    ltl_opts o;
    memset(&o, 0, sizeof o);
    o.stop_on_solution = LTL_STOP_FIRST;
    return o;
}

// Runs one problem to completion in slot 0 of engine e (the whole workspace).
ltl_status run_single(Engine &e, ProblemIn &&in, char *formula_out, size_t formula_cap, ltl_stats *stats) {
    const double t0 = wall_ms();
    if (formula_out && formula_cap) formula_out[0] = '\0';
    // the previous problem of a context is kept until the next call
    if (e.slots[0].state != SLOT_FREE) e.release(0);
    // size the workspace for this problem's fixed part (and let it grow)
    Layout probe;
    ltl_status s = plan_layout(in, e.opts.max_chunks, e.opts.level_kernel, 0, (uint64_t)1 << 62, probe);
    if (s != LTL_OK) return s;
    const size_t fixed = probe.o_hslots + (1 << 20);
    s = e.ensure_workspace(e.shared_end + fixed + (e.opts.mem_budget_bytes ? e.opts.mem_budget_bytes : 0));
    if (s != LTL_OK) return s;
    uint64_t budget = e.opts.mem_budget_bytes;
    if (e.opts.workspace && e.opts.mem_budget_bytes) budget = std::min<uint64_t>(budget, e.mem.largest());
    s = e.admit(0, in, budget);
    if (s != LTL_OK) return s;
    while (e.slots[0].state == SLOT_RUNNING) {
        s = e.round();
        if (s != LTL_OK) return s;
    }
    Slot &sl = e.slots[0];
    sl.st.total_ms = wall_ms() - t0;
    if (stats) *stats = sl.st;
    if (sl.status < 0) return fail(sl.status, "%s", sl.error.c_str());
    if (sl.status == LTL_OK) {
        s = write_formula(sl.formula, formula_out, formula_cap);
        if (s != LTL_OK) return s;
    }
    return sl.status;
}

// ============================================================= BatchRunner

struct BatchRunner {
    Engine e;
    std::deque<ProblemIn> queue;
    uint64_t share = 0;
};

ltl_status runner_create(const ltl_opts &o, int max_resident, int share_divisor, BatchRunner **out) {
    *out = nullptr;
    std::unique_ptr<BatchRunner> r(new BatchRunner());
    ltl_status s = r->e.setup(&o, max_resident, false);
    if (s != LTL_OK) return s;
    s = r->e.ensure_workspace(r->e.shared_end + ((size_t)64 << 20));
    if (s != LTL_OK) return s;
    r->share = (r->e.ws_bytes - r->e.shared_end) / (uint64_t)std::max(1, share_divisor);
    *out = r.release();
    return LTL_OK;
}

void runner_destroy(BatchRunner *r) { delete r; }

ltl_status runner_submit(BatchRunner *r, const ltl_traces &P, const ltl_traces &N, int n_props, uint32_t ops,
                         int max_size, uint64_t budget, uint64_t id, bool copy) {
    ProblemIn in;
    ltl_status s = problem_from_host(&P, &N, n_props, ops, max_size, budget, copy, in);
    if (s != LTL_OK) return s;
    in.id = id;
    r->queue.push_back(std::move(in));
    return LTL_OK;
}

ltl_status runner_step(BatchRunner *r, std::vector<ltl_result> &done) {
    Engine &e = r->e;
    // admit in order while memory and slots allow
    while (!r->queue.empty()) {
        int si = -1;
        for (int j = 0; j < e.max_slots; ++j)
            if (e.slots[j].state == SLOT_FREE) {
                si = j;
                break;
            }
        if (si < 0) break;
        ProblemIn &front = r->queue.front();
        const uint64_t budget = front.budget ? front.budget : r->share;
        const ltl_status as = e.admit(si, front, budget);
        if (as == LTL_OK) {
            r->queue.pop_front();
            continue;
        }
        if (as == LTL_ERR_OOM && e.resident() > 0) break;   // wait for memory
        ltl_result res;                                     // does not fit even alone, or invalid
        memset(&res, 0, sizeof res);
        res.id = front.id;
        res.status = as;
        done.push_back(res);
        r->queue.pop_front();
    }
    if (e.resident() == 0) return LTL_OK;
    ltl_status s = e.round();
    if (s != LTL_OK) return s;
    for (int j = 0; j < e.max_slots; ++j) {
        Slot &sl = e.slots[j];
        if (sl.state != SLOT_DONE) continue;
        ltl_result res;
        e.fill_result(sl, res);
        done.push_back(res);
        e.release(j);
    }
    return LTL_OK;
}

bool runner_busy(const BatchRunner *r) { return !r->queue.empty() || r->e.resident() > 0; }
cudaStream_t runner_stream(const BatchRunner *r) { return r->e.stream; }
uint64_t runner_rounds(const BatchRunner *r) { return r->e.total_rounds; }

}  // namespace ltl

using namespace ltl;

// ==================================================================== C ABI

struct ltl_ctx {
    Engine e;
};

struct ltl_server {
    Engine e;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<ProblemIn> queue;
    std::deque<ltl_result> done;
    std::thread worker;
    bool stop = false;
    uint64_t next_id = 0;
    uint64_t default_budget = 0;
    ltl_status worker_error = LTL_OK;
    std::string worker_msg;
};

extern "C" {

ltl_status ltl_ctx_create(const ltl_opts *opts, ltl_ctx **out) {
    if (!out) return fail(LTL_ERR_INVALID, "out is NULL");
    *out = nullptr;
    const ltl_opts o = opts ? *opts : default_opts();
    if (o.stop_on_solution < 0 || o.stop_on_solution > 2) return fail(LTL_ERR_INVALID, "stop_on_solution must be 0, 1 or 2");
    ltl_ctx *c = new ltl_ctx();
    ltl_status s = c->e.setup(&o, 1, true);
    if (s != LTL_OK) {
        delete c;
        return s;
    }
    *out = c;
    return LTL_OK;
}

void ltl_ctx_destroy(ltl_ctx *c) { delete c; }

ltl_status ltl_ctx_set_mem_budget(ltl_ctx *c, uint64_t bytes) {
    if (!c) return fail(LTL_ERR_INVALID, "ctx is NULL");
    c->e.opts.mem_budget_bytes = bytes;
    return LTL_OK;
}

ltl_status ltl_ctx_learn(ltl_ctx *c, const ltl_traces *P, const ltl_traces *N, int n_props, uint32_t ops,
                         int max_size, char *formula_out, size_t formula_cap, ltl_stats *stats) {
    if (!c) return fail(LTL_ERR_INVALID, "ctx is NULL");
    ProblemIn in;
    ltl_status s = problem_from_host(P, N, n_props, ops, max_size, 0, false, in);
    if (s != LTL_OK) return s;
    return run_single(c->e, std::move(in), formula_out, formula_cap, stats);
}

ltl_status ltl_ctx_learn_device(ltl_ctx *c, const uint32_t *d_letters, const uint64_t *d_offsets, uint64_t n_pos,
                                uint64_t n_neg, uint32_t max_len, int n_props, uint32_t ops, int max_size,
                                char *formula_out, size_t formula_cap, ltl_stats *stats) {
    if (!c) return fail(LTL_ERR_INVALID, "ctx is NULL");
    ltl_status s = check_common(n_props, ops, max_size);
    if (s != LTL_OK) return s;
    if (!d_offsets || (!d_letters && max_len > 0)) return fail(LTL_ERR_INVALID, "device trace buffers are NULL");
    ProblemIn in;
    in.device_input = true;
    in.d_letters = d_letters;
    in.d_offsets = d_offsets;
    in.n_pos = n_pos;
    in.n_neg = n_neg;
    in.max_len = max_len;
    in.n_props = n_props;
    in.ops = ops;
    in.max_size = max_size;
    in.t_submit = wall_ms();
    return run_single(c->e, std::move(in), formula_out, formula_cap, stats);
}

ltl_status ltl_learn(const ltl_traces *P, const ltl_traces *N, int n_props, uint32_t ops, int max_size,
                     const ltl_opts *opts, char *formula_out, size_t formula_cap, ltl_stats *stats) {
    ltl_ctx *c = nullptr;
    ltl_status s = ltl_ctx_create(opts, &c);
    if (s != LTL_OK) return s;
    s = ltl_ctx_learn(c, P, N, n_props, ops, max_size, formula_out, formula_cap, stats);
    ltl_ctx_destroy(c);
    return s;
}

ltl_status ltl_ctx_autotune_dump(ltl_ctx *c, char *out, size_t cap, size_t *needed) {
    if (!c) return fail(LTL_ERR_INVALID, "ctx is NULL");
    const std::string text = c->e.tuner.dump();
    if (needed) *needed = text.size() + 1;
    return write_formula(text, out, cap);
}

ltl_status ltl_ctx_level_range(ltl_ctx *c, int level, uint64_t *begin, uint64_t *count) {
    if (!c || !begin || !count) return fail(LTL_ERR_INVALID, "NULL argument");
    const Slot &s = c->e.slots[0];
    if (s.state != SLOT_DONE) return fail(LTL_ERR_INVALID, "no learn result on this context");
    if (level < 1 || level >= kMaxLevels) return fail(LTL_ERR_INVALID, "level out of range");
    *begin = s.lvl_begin[level];
    *count = s.lvl_count[level];
    return LTL_OK;
}

ltl_status ltl_ctx_entry(ltl_ctx *c, uint64_t idx, char *formula_out, size_t formula_cap, uint64_t *cs_out,
                         int words_per_trace) {
    if (!c) return fail(LTL_ERR_INVALID, "ctx is NULL");
    Engine &e = c->e;
    const Slot &s = e.slots[0];
    if (s.state != SLOT_DONE) return fail(LTL_ERR_INVALID, "no learn result on this context");
    const Layout &L = s.L;
    if (idx >= s.prev_entries) return fail(LTL_ERR_INVALID, "entry %llu out of range", (unsigned long long)idx);
    if (formula_out) {
        std::string text;
        ltl_status st = e.entry_formula(0, idx, text);
        if (st != LTL_OK) return st;
        if ((st = write_formula(text, formula_out, formula_cap)) != LTL_OK) return st;
    }
    if (!cs_out) return LTL_OK;
    const char *src = e.ws + s.off + L.o_arena + 8 * L.stride * idx;
    if (L.narrow) {
        if (words_per_trace != 1) return fail(LTL_ERR_INVALID, "words_per_trace must be 1");
        // word q of the plane holds traces 2q (low half) and 2q + 1 (high half)
        const uint64_t nw = ((uint64_t)L.n_traces + 1) / 2;
        std::vector<uint64_t> words(nw ? nw : 1);
        LTL_CUDA_TRY(cudaMemcpyAsync(words.data(), src, 8 * nw, cudaMemcpyDeviceToHost, e.stream));
        LTL_CUDA_TRY(cudaStreamSynchronize(e.stream));
        for (uint64_t t = 0; t < L.n_traces; ++t) cs_out[t] = (words[t / 2] >> (32 * (t & 1))) & 0xffffffffull;
        return LTL_OK;
    }
    if (words_per_trace != L.W) return fail(LTL_ERR_INVALID, "words_per_trace must be %d", L.W);
    // plane w of the entry holds word w of every trace: a strided 2-D copy
    for (int w = 0; w < L.W; ++w)
        LTL_CUDA_TRY(cudaMemcpy2DAsync(cs_out + w, 8 * (size_t)L.W, src + 8 * L.plane * w, 8, 8, (size_t)L.n_traces,
                                       cudaMemcpyDeviceToHost, e.stream));
    LTL_CUDA_TRY(cudaStreamSynchronize(e.stream));
    return LTL_OK;
}

ltl_status ltl_learn_batch(int n, const ltl_problem *problems, const ltl_opts *opts, ltl_result *out) {
    if (n < 0 || (n > 0 && (!problems || !out))) return fail(LTL_ERR_INVALID, "bad batch arguments");
    if (n == 0) return LTL_OK;
    const ltl_opts o = opts ? *opts : default_opts();
    if (o.stop_on_solution < 0 || o.stop_on_solution > 2) return fail(LTL_ERR_INVALID, "stop_on_solution must be 0, 1 or 2");
    const int resident_cap = std::min(n, 1024);
    BatchRunner *r = nullptr;
    ltl_status s = runner_create(o, resident_cap, resident_cap, &r);
    if (s != LTL_OK) return s;
    std::unique_ptr<BatchRunner, void (*)(BatchRunner *)> guard(r, runner_destroy);
    // problems are queued in input order; each needs its budget (or an equal
    // share of the workspace) of contiguous memory to be admitted
    for (int i = 0; i < n; ++i) {
        const ltl_problem &p = problems[i];
        memset(&out[i], 0, sizeof(ltl_result));
        out[i].id = (uint64_t)i;
        s = runner_submit(r, p.P, p.N, p.n_props, p.ops, p.max_size, p.mem_budget_bytes, (uint64_t)i, false);
        if (s != LTL_OK) out[i].status = s;
    }
    std::vector<ltl_result> done;
    while (runner_busy(r)) {
        s = runner_step(r, done);
        if (s != LTL_OK) return s;
        for (const ltl_result &d : done) out[d.id] = d;
        done.clear();
    }
    return LTL_OK;
}

static void server_loop(ltl_server *srv) {
    cudaSetDevice(srv->e.device);
    Engine &e = srv->e;
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(srv->mu);
            srv->cv_work.wait(lk, [&] { return srv->stop || !srv->queue.empty() || e.resident() > 0; });
            if (srv->stop) return;
            // admission between rounds: in arrival order, while memory fits
            while (!srv->queue.empty()) {
                int si = -1;
                for (int j = 0; j < e.max_slots; ++j)
                    if (e.slots[j].state == SLOT_FREE) {
                        si = j;
                        break;
                    }
                if (si < 0) break;
                ProblemIn &front = srv->queue.front();
                const uint64_t id = front.id;
                const double t_sub = front.t_submit;
                const uint64_t budget = front.budget ? front.budget : srv->default_budget;
                ltl_status as = e.admit(si, front, budget);
                if (as == LTL_OK) {
                    srv->queue.pop_front();
                    continue;
                }
                if (as == LTL_ERR_OOM && e.resident() > 0) break;   // wait for memory
                ltl_result r;
                memset(&r, 0, sizeof r);
                r.id = id;
                r.status = as;
                r.latency_ms = wall_ms() - t_sub;
                srv->queue.pop_front();
                srv->done.push_back(r);
                srv->cv_done.notify_all();
            }
        }
        if (e.resident() == 0) continue;
        ltl_status s = e.round();
        std::lock_guard<std::mutex> lk(srv->mu);
        if (s != LTL_OK) {
            srv->worker_error = s;
            srv->worker_msg = "round failed";
            // fail every resident problem
            for (int j = 0; j < e.max_slots; ++j)
                if (e.slots[j].state == SLOT_RUNNING) e.finish(e.slots[j], s);
        }
        for (int j = 0; j < e.max_slots; ++j) {
            Slot &sl = e.slots[j];
            if (sl.state != SLOT_DONE) continue;
            ltl_result r;
            e.fill_result(sl, r);
            srv->done.push_back(r);
            e.release(j);
        }
        srv->cv_done.notify_all();
    }
}

ltl_status ltl_server_create(const ltl_opts *opts, int max_resident, ltl_server **out) {
    if (!out) return fail(LTL_ERR_INVALID, "out is NULL");
    *out = nullptr;
    const ltl_opts o = opts ? *opts : default_opts();
    if (max_resident < 1 || max_resident > 4096) return fail(LTL_ERR_INVALID, "max_resident must be in 1..4096");
    ltl_server *srv = new ltl_server();
    ltl_status s = srv->e.setup(&o, max_resident, false);
    if (s == LTL_OK) s = srv->e.ensure_workspace(srv->e.shared_end + ((size_t)64 << 20));
    if (s != LTL_OK) {
        delete srv;
        return s;
    }
    srv->default_budget = (srv->e.ws_bytes - srv->e.shared_end) / (uint64_t)max_resident;
    if (o.mem_budget_bytes) srv->default_budget = o.mem_budget_bytes;
    srv->worker = std::thread(server_loop, srv);
    *out = srv;
    return LTL_OK;
}

ltl_status ltl_server_submit(ltl_server *srv, const ltl_problem *p, uint64_t *id) {
    if (!srv || !p) return fail(LTL_ERR_INVALID, "NULL argument");
    ProblemIn in;
    ltl_status s = problem_from_host(&p->P, &p->N, p->n_props, p->ops, p->max_size, p->mem_budget_bytes, true, in);
    if (s != LTL_OK) return s;
    std::lock_guard<std::mutex> lk(srv->mu);
    in.id = srv->next_id++;
    if (id) *id = in.id;
    srv->queue.push_back(std::move(in));
    srv->cv_work.notify_all();
    return LTL_OK;
}

ltl_status ltl_server_poll(ltl_server *srv, ltl_result *out, int max, int *n_out, int wait_ms) {
    if (!srv || !n_out || (max > 0 && !out)) return fail(LTL_ERR_INVALID, "NULL argument");
    std::unique_lock<std::mutex> lk(srv->mu);
    if (srv->done.empty() && wait_ms > 0)
        srv->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), [&] { return !srv->done.empty(); });
    int n = 0;
    while (n < max && !srv->done.empty()) {
        out[n++] = srv->done.front();
        srv->done.pop_front();
    }
    *n_out = n;
    if (srv->worker_error != LTL_OK && n == 0) return fail(srv->worker_error, "%s", srv->worker_msg.c_str());
    return LTL_OK;
}

ltl_status ltl_server_pending(ltl_server *srv, uint64_t *queued, uint64_t *resident) {
    if (!srv) return fail(LTL_ERR_INVALID, "NULL argument");
    std::lock_guard<std::mutex> lk(srv->mu);
    if (queued) *queued = srv->queue.size();
    if (resident) *resident = (uint64_t)srv->e.resident();
    return LTL_OK;
}

void ltl_server_destroy(ltl_server *srv) {
    if (!srv) return;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
        srv->cv_work.notify_all();
    }
    if (srv->worker.joinable()) srv->worker.join();
    delete srv;
}

}  // extern "C"
