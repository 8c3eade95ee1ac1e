/*
 * gputf_utf16_to_utf8_static: the UTF-16 -> UTF-8 transcoder without a
 * caller-provided workspace.
 *
 * Who needs it: code that must not allocate device memory when it runs.
 * Examples are a library call made while a stream is being captured into a
 * CUDA graph in a mode that forbids cudaMalloc, code running inside a custom
 * allocator or memory-pool callback (allocating there would re-enter the
 * allocator), and services that reserve all their device memory at start-up
 * and may not allocate afterwards.  Such a caller still owns the input, the
 * output and the result; only the scratch moves into the library.
 *
 * The scratch (the tile-status words and counters the transcoder uses) is a
 * fixed array in this file.  Every GPU that loads the library holds its own
 * copy until the process exits.  It is sized for inputs of up to
 * GPUTF_STATIC_MAX_UNITS units; larger inputs are refused.
 */
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include "gputf.h"
#include "common.cuh"
#include "kernels.h"

namespace {

/* Same sizing rule as gputf_workspace_bytes(): a header plus one status word
 * per 1024 units (tiles are never smaller than that), plus two. */
constexpr size_t STATIC_SCRATCH_BYTES =
    gputf::HEADER_BYTES + 8 * ((GPUTF_STATIC_MAX_UNITS + 16) / 1024 + 2);

static __device__ __align__(256) unsigned char g_static_scratch[STATIC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;

struct StaticScratch {
    bool ready = false;
    void *ptr = nullptr;   /* device address of g_static_scratch on this device */
};

StaticScratch g_scratch[MAX_DEVICES];
std::mutex g_scratch_mutex;

}  // namespace

extern "C" gputf_status gputf_utf16_to_utf8_static(const uint16_t *in, size_t n_units, uint8_t *out,
                                                   size_t out_cap, gputf_result *res,
                                                   cudaStream_t stream)
{
    if ((uint64_t)n_units > GPUTF_STATIC_MAX_UNITS) return GPUTF_STATUS_INPUT_TOO_LARGE;
    if ((n_units > 0 && in == nullptr) || res == nullptr || (out_cap > 0 && out == nullptr) ||
        ((uintptr_t)in & 1) || ((uintptr_t)res & 7))
        return GPUTF_STATUS_INVALID_ARGUMENT;   /* refused before the set-up below touches the GPU */

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES)
        return GPUTF_STATUS_CUDA_ERROR;
    void *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_scratch_mutex);
        StaticScratch &st = g_scratch[dev];
        if (!st.ready) {
            /* set-up, once per device, with that device current: the array's
             * device address (the host-side symbol is not one), then the
             * scratch is put in its starting state on the caller's stream.
             * On a stream being captured that state would only be recorded,
             * not reached, so the set-up is refused there. */
            cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
            if (cudaStreamIsCapturing(stream, &cap) != cudaSuccess) return GPUTF_STATUS_CUDA_ERROR;
            if (cap != cudaStreamCaptureStatusNone) return GPUTF_STATUS_INVALID_ARGUMENT;
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || p == nullptr)
                return GPUTF_STATUS_CUDA_ERROR;
            if (gputf::launch_workspace_init(p, STATIC_SCRATCH_BYTES, stream) != cudaSuccess)
                return GPUTF_STATUS_CUDA_ERROR;
            st.ptr = p;
            st.ready = true;
        }
        scratch = st.ptr;
    }
    return gputf_utf16_to_utf8(in, n_units, out, out_cap, scratch, STATIC_SCRATCH_BYTES, res, stream);
}
