/*
 * gputf_test_wait_timeout: drives one of the kernels' bounded waits to its
 * limit on purpose, so that a test can check that a wait that never ends
 * comes back as GPUTF_TIMEOUT with the GPU still usable.  Nothing faults and
 * nothing hangs: the waits are the kernels' own (look_back and mbar_wait of
 * common.cuh) with a small poll limit, and they simply run out.
 *
 *   which = 0: one warp runs the decoupled look-back of tile 1 of a call in
 *              the workspace's current epoch; tile 0 never publishes, so every
 *              poll of its status word finds an older epoch;
 *   which = 1: one thread waits on a shared-memory mbarrier that expects one
 *              arrival which never comes (no copy is issued, so none is in
 *              flight when the block exits).
 * The result and the end of the call are the transcoders' own: the timeout
 * recorded in the workspace header becomes GPUTF_TIMEOUT, and the header is
 * reset for the next call as every kernel's last block does.
 */
#include <cstdint>

#include <cuda_runtime.h>

#include "gputf.h"
#include "common.cuh"
#include "kernels.h"

namespace {

__global__ void wait_timeout_kernel(gputf::WsHeader *hdr, unsigned long long *status, uint64_t status_words,
                                    int which, int polls, gputf::DevResult *res)
{
    using namespace gputf;
    __shared__ unsigned long long s_bar;
    __shared__ unsigned s_flag;
    const unsigned epoch = *(volatile unsigned *)&hdr->epoch;
    if (which == 0) {
        if (threadIdx.x < 32) look_back(status, 1, epoch, &hdr->flags, polls);
    } else {
        if (threadIdx.x == 0) {
            mbar_init(&s_bar, 1);
            fence_mbar_init();
            if (!mbar_wait(&s_bar, 0, polls)) atomicOr(&hdr->flags, FLAG_TIMEOUT);
        }
    }
    if (!finish_cta(hdr, &s_flag)) return;
    if (threadIdx.x == 0) {
        const unsigned flags = *(volatile unsigned *)&hdr->flags;
        res->error = (flags & FLAG_TIMEOUT) ? GPUTF_E_TIMEOUT : GPUTF_E_OK;
        res->reserved = 0;
        res->position = 0;
        res->written = 0;
    }
    reset_workspace(hdr, status, status_words);
}

}  // namespace

extern "C" gputf_status gputf_test_wait_timeout(void *ws, size_t ws_bytes, int which, uint32_t polls,
                                                gputf_result *res, cudaStream_t stream)
{
    if (ws == nullptr || res == nullptr || ((uintptr_t)ws & 15) || ((uintptr_t)res & 7) ||
        ws_bytes < gputf::HEADER_BYTES + 8 || (which != 0 && which != 1) || polls == 0 || polls > (1u << 20))
        return GPUTF_STATUS_INVALID_ARGUMENT;
    auto *hdr = static_cast<gputf::WsHeader *>(ws);
    auto *status = reinterpret_cast<unsigned long long *>(static_cast<char *>(ws) + gputf::HEADER_BYTES);
    const uint64_t words = (ws_bytes - gputf::HEADER_BYTES) / 8;
    wait_timeout_kernel<<<1, 32, 0, stream>>>(hdr, status, words, which, (int)polls,
                                              reinterpret_cast<gputf::DevResult *>(res));
    return gputf::status_of(cudaGetLastError());
}
