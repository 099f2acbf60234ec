// ltl_internal.h -- host-side declarations shared by the library's translation
// units (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "ltl.h"
#include "ltl_types.h"

namespace ltl {

// ---- errors: message of the last failure on this host thread
ltl_status fail(ltl_status s, const char *fmt, ...);
ltl_status set_error(ltl_status s, const char *msg);

#define LTL_CUDA_TRY(x)                                                                      \
    do {                                                                                     \
        cudaError_t e_ = (x);                                                                \
        if (e_ != cudaSuccess) {                                                             \
            (void)cudaGetLastError();                                                        \
            return ::ltl::fail(LTL_ERR_CUDA, "%s failed: %s", #x, cudaGetErrorString(e_));   \
        }                                                                                    \
    } while (0)

inline uint64_t round_up(uint64_t x, uint64_t m) { return (x + m - 1) / m * m; }
inline uint64_t pow2_ceil(uint64_t x) {
    uint64_t p = 1;
    while (p < x) p <<= 1;
    return p;
}
inline int ceil_log2(uint64_t x) {   // smallest k with 2^k >= x (0 for x <= 1)
    int k = 0;
    while ((1ull << k) < x) ++k;
    return k;
}
double wall_ms();

// ---- formula text
bool compile_formula(const char *text, int n_props, std::vector<uint32_t> &prog, int &depth, int &max_atom);
bool compile_formula_program(const char *text, int n_props, std::vector<uint32_t> &prog, int &depth);
size_t tokens_to_text(const uint32_t *tok, int n, int i, std::string &out);
ltl_status write_formula(const std::string &s, char *out, size_t cap);
ltl_status check_common(int n_props, uint32_t ops, int max_size);
ltl_status check_traces(const ltl_traces *t, const char *name);
uint64_t traces_max_len(const ltl_traces *t);

// ---- batch runner: an engine that advances queued learning problems one
// level per round, with launches shared between the resident problems
// (continuous batching; used by ltl_learn_batch and divide and conquer)
struct BatchRunner;
// `share_divisor`: a problem without its own budget gets this fraction of the
// workspace left after the shared region
ltl_status runner_create(const ltl_opts &o, int max_resident, int share_divisor, BatchRunner **out);
void runner_destroy(BatchRunner *r);
// queues a problem; the traces are copied when `copy`, else they must stay
// valid until its result comes back; `id` comes back in its result
ltl_status runner_submit(BatchRunner *r, const ltl_traces &P, const ltl_traces &N, int n_props, uint32_t ops,
                         int max_size, uint64_t budget, uint64_t id, bool copy);
// admits queued problems while slots and memory allow, runs one round, and
// appends the results of the problems that finished (or could not be admitted)
ltl_status runner_step(BatchRunner *r, std::vector<ltl_result> &done);
bool runner_busy(const BatchRunner *r);
cudaStream_t runner_stream(const BatchRunner *r);
uint64_t runner_rounds(const BatchRunner *r);

// ---- kernels (device code lives in the other translation units)
const void *fused_kernel_ptr_w1(int C, int op);
const void *fused_kernel_ptr_w2(int C, int op);
const void *fused_kernel_ptr_w48(int W, int C, int op);
const void *fused_kernel_ptr_narrow(int C, int op);
const void *stream_kernel_ptr(int W, int C);
size_t stream_smem_bytes(int W, int C, int NT);   // the streaming kernel's operand ring
const void *cluster_kernel_ptr(int W, int C);
int fused_kernel_batch(int W, int C, bool narrow);
const void *ws_kernel_ptr_w1(int C, int op);
const void *ws_kernel_ptr_wn(int W, int C, int op);
const void *ws_kernel_ptr_narrow(int C, int op);
int ws_kernel_batch(int W, int C, bool narrow);
constexpr int kWsExtraThreads = 64;   // the hash warps of a warp-specialised level kernel
inline const void *fused_kernel_ptr(int W, int C, int op) {
    return W == 1 ? fused_kernel_ptr_w1(C, op) : W == 2 ? fused_kernel_ptr_w2(C, op) : fused_kernel_ptr_w48(W, C, op);
}

// Trace packing: traces of at most 64 * W positions into Wt >= W words each
// (all Wt planes written); with `keys` also the NH fingerprint keys of `seed`,
// one per matrix word (Wt * plane words, the stride of one matrix); with
// `zero` (16-byte aligned) the same launch also clears n_zero16 16-byte units
// there.
cudaError_t launch_pack(const uint32_t *letters, const uint64_t *offsets, uint32_t n_traces, uint64_t plane, int W,
                        int Wt, int n_props, uint64_t *mask, uint64_t *atoms, uint64_t stride, Ctrl *ctrl,
                        cudaStream_t s, uint64_t *keys = nullptr, uint64_t seed = 0, void *zero = nullptr,
                        uint64_t n_zero16 = 0);
cudaError_t launch_pack_narrow(const uint32_t *letters, const uint64_t *offsets, uint32_t n_traces, uint64_t plane,
                               int n_props, uint64_t *mask, uint64_t *atoms, uint64_t stride, Ctrl *ctrl,
                               cudaStream_t s, uint64_t *keys = nullptr, uint64_t seed = 0, void *zero = nullptr,
                               uint64_t n_zero16 = 0);
cudaError_t launch_walk_batch(const WalkJob *jobs, int n_jobs, uint32_t *tokens, int cap, int *n_out, cudaStream_t s);
struct PlanArgs;
cudaError_t launch_plan(const PlanArgs &a, int k, bool close_prev, bool plan_this, cudaStream_t s);
cudaError_t launch_eval(int W, const uint32_t *prog, int n_instr, const uint64_t *atoms, const uint64_t *mask,
                        uint64_t stride, uint64_t plane, uint64_t *stack, int nsteps, uint32_t n_traces,
                        uint64_t *out, int out_words, cudaStream_t s);

}  // namespace ltl
