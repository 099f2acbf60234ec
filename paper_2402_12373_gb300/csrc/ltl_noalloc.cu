// ltl_noalloc.cu -- ltl_eval without any device allocation.
//
// Some callers cannot allocate device memory at all: code running inside a
// framework that owns every byte of the device through its own pool,
// real-time or safety-critical loops where allocation is forbidden after
// start-up, or code that must not trigger the implicit synchronisation that
// cudaMalloc / cudaFree cause.  For them this file offers one entry point that
// evaluates a formula exactly like ltl_eval, but on device-resident traces,
// writing a device-resident result, with all intermediate storage taken from
// one file-scope static device array of a fixed size.
//
// Properties of that array (documented again in include/ltl.h):
//  * its size is kNoallocScratchBytes (64 MiB); every GPU that loads this
//    library holds it until the process exits;
//  * every call on a device shares it and it keeps the last call's contents;
//    the parts that must start at zero are cleared by each call, on the
//    caller's stream; two calls whose work overlaps on the GPU (different
//    streams, or different host threads) race on it and must be serialised by
//    the caller;
//  * its device address is looked up once per device, by the first call on
//    that device (cudaGetSymbolAddress, with that device current);
//  * every call reads a status word back into host memory and synchronises
//    the stream, so no call can be made while a stream is being captured.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "ltl_internal.h"

namespace {

constexpr size_t kNoallocScratchBytes = (size_t)LTL_NOALLOC_SCRATCH_BYTES;

// The scratch memory of every ltl_eval_noalloc call on this device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of the static scratch on the current device (set-up once per
// device; the symbol's name in host code is only a host-side handle).
ltl_status scratch_on_current_device(unsigned char **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return ltl::set_error(LTL_ERR_CUDA, "ltl_eval_noalloc: no current CUDA device");
    }
    if (dev < 0 || dev >= kMaxDevices) return ltl::set_error(LTL_ERR_INVALID, "ltl_eval_noalloc: device index too large");
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            (void)cudaGetLastError();
            return ltl::set_error(LTL_ERR_CUDA, "ltl_eval_noalloc: cudaGetSymbolAddress of the static scratch failed");
        }
        g_scratch_ptr[dev] = p;
    }
    *out = (unsigned char *)g_scratch_ptr[dev];
    return LTL_OK;
}

}  // namespace

extern "C" ltl_status ltl_eval_noalloc(const char *formula, const uint32_t *d_letters, const uint64_t *d_offsets,
                                       uint64_t n_traces, uint32_t max_len, int n_props, uint64_t *d_cs_out,
                                       int words_per_trace, void *stream) {
    using namespace ltl;
    if (n_props < 1 || n_props > 32) return set_error(LTL_ERR_INVALID, "ltl_eval_noalloc: n_props must be in 1..32");
    if (n_traces > 0x7fffffffull) return set_error(LTL_ERR_INVALID, "ltl_eval_noalloc: too many traces");
    if (!d_offsets || (n_traces && !d_cs_out) || (max_len && !d_letters))
        return set_error(LTL_ERR_INVALID, "ltl_eval_noalloc: NULL device buffer");
    std::vector<uint32_t> prog;
    int depth = 0;
    if (!compile_formula_program(formula, n_props, prog, depth))
        return set_error(LTL_ERR_INVALID, "ltl_eval_noalloc: cannot parse formula (or an atom >= n_props)");
    const int W = (int)((max_len + 63) / 64 > 0 ? (max_len + 63) / 64 : 1);
    int Wt = 1;
    while (Wt < W) Wt <<= 1;
    if (Wt > 16) return set_error(LTL_ERR_INVALID, "ltl_eval_noalloc: traces up to 1024 positions are supported");
    if (words_per_trace < W) return set_error(LTL_ERR_INVALID, "ltl_eval_noalloc: words_per_trace too small");
    if (n_traces == 0) return LTL_OK;
    const uint64_t plane = ltl::round_up(n_traces, 128), stride = (uint64_t)Wt * plane;
    // scratch layout: control block | program | masks | atoms | operand stack
    const uint64_t o_ctrl = 0;
    const uint64_t o_prog = ltl::round_up(sizeof(Ctrl), 256);
    const uint64_t o_mask = ltl::round_up(o_prog + 4 * prog.size(), 256);
    const uint64_t o_atoms = ltl::round_up(o_mask + 8 * stride, 256);
    const uint64_t o_stack = ltl::round_up(o_atoms + 8 * stride * (uint64_t)n_props, 256);
    const uint64_t need = o_stack + 8 * stride * (uint64_t)depth;
    if (need > kNoallocScratchBytes) {
        char msg[256];
        snprintf(msg, sizeof msg,
                 "ltl_eval_noalloc: this evaluation needs %llu bytes of scratch; the static scratch holds %llu "
                 "(LTL_NOALLOC_SCRATCH_BYTES)",
                 (unsigned long long)need, (unsigned long long)kNoallocScratchBytes);
        return set_error(LTL_ERR_OOM, msg);
    }
    unsigned char *scr = nullptr;
    ltl_status st = scratch_on_current_device(&scr);
    if (st != LTL_OK) return st;
    cudaStream_t sm = (cudaStream_t)stream;
    Ctrl *ctrl = (Ctrl *)(scr + o_ctrl);
    uint64_t *mask = (uint64_t *)(scr + o_mask);
    uint64_t *atoms = (uint64_t *)(scr + o_atoms);
#define NOALLOC_TRY(x)                                                                 \
    do {                                                                               \
        cudaError_t e_ = (x);                                                          \
        if (e_ != cudaSuccess) {                                                       \
            (void)cudaGetLastError();                                                  \
            std::string m_ = std::string("ltl_eval_noalloc: ") + #x + ": " + cudaGetErrorString(e_); \
            return set_error(LTL_ERR_CUDA, m_.c_str());                                \
        }                                                                              \
    } while (0)
    // what must start at zero: the control word (the pack kernel writes every
    // word of the mask and atom planes, padding planes and traces included)
    NOALLOC_TRY(cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), sm));
    NOALLOC_TRY(cudaMemcpyAsync(scr + o_prog, prog.data(), 4 * prog.size(), cudaMemcpyHostToDevice, sm));
    NOALLOC_TRY(launch_pack(d_letters, d_offsets, (uint32_t)n_traces, plane, W, Wt, n_props, mask, atoms, stride, ctrl, sm));
    // log steps for the packed capacity (64 * W positions), not for max_len:
    // the pack kernel accepts any trace that fits W words, and a trace longer
    // than max_len evaluated with max_len's steps would lose the F / G / U
    // bits beyond 2^steps (extra steps are harmless)
    int nsteps = 0;
    while ((1ull << nsteps) < 64ull * (uint64_t)W) ++nsteps;
    NOALLOC_TRY(launch_eval(Wt, (const uint32_t *)(scr + o_prog), (int)prog.size(), atoms, mask, stride, plane,
                            (uint64_t *)(scr + o_stack), nsteps, (uint32_t)n_traces, d_cs_out, words_per_trace, sm));
    int invalid = 0;
    NOALLOC_TRY(cudaMemcpyAsync(&invalid, &ctrl->invalid_letter, sizeof(int), cudaMemcpyDeviceToHost, sm));
    NOALLOC_TRY(cudaStreamSynchronize(sm));
#undef NOALLOC_TRY
    if (invalid)
        return set_error(LTL_ERR_INVALID,
                         "ltl_eval_noalloc: letters use propositions >= n_props, offsets decrease, or a trace is "
                         "longer than 64 * ceil(max_len / 64) positions");
    return LTL_OK;
}
