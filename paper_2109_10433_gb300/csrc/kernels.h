/* Internal interface between the C-ABI layer (api.cu) and the kernels. */
#ifndef GPUTF_KERNELS_H
#define GPUTF_KERNELS_H

#include <cstdint>
#include <cuda_runtime.h>

#include "gputf.h"

namespace gputf {

/* Same layout as gputf_result in the public header. */
struct DevResult {
    int32_t error;
    int32_t reserved;
    uint64_t position;
    uint64_t written;
};

uint64_t utf8_to_utf16_tiles(const void *in, uint64_t n);
uint64_t utf16_to_utf8_tiles(const void *in, uint64_t n);

cudaError_t launch_utf8_to_utf16(const uint8_t *in, uint64_t n, uint16_t *out, uint64_t cap,
                                 void *ws, uint64_t status_words, DevResult *res, int sms, bool validate,
                                 bool big_endian, bool chained, cudaStream_t s);
cudaError_t launch_utf16_to_utf8(const uint16_t *in, uint64_t n, uint8_t *out, uint64_t cap,
                                 void *ws, uint64_t status_words, DevResult *res, int sms, bool validate,
                                 bool big_endian, bool chained, cudaStream_t s);
cudaError_t launch_validate_utf8(const uint8_t *in, uint64_t n, void *ws, DevResult *res, int sms,
                                 cudaStream_t s);
cudaError_t launch_validate_utf16(const uint16_t *in, uint64_t n, void *ws, DevResult *res, int sms,
                                  bool big_endian, cudaStream_t s);
cudaError_t launch_utf16_length_from_utf8(const uint8_t *in, uint64_t n, void *ws,
                                          unsigned long long *len, int sms, cudaStream_t s);
cudaError_t launch_utf8_length_from_utf16(const uint16_t *in, uint64_t n, void *ws,
                                          unsigned long long *len, int sms, bool big_endian, cudaStream_t s);
cudaError_t launch_workspace_init(void *ws, uint64_t bytes, cudaStream_t s);

/* A CUDA error as a call status, recorded for gputf_last_cuda_error (api.cu). */
gputf_status status_of(cudaError_t e);

/* Span gather (gather.cu). */
cudaError_t launch_gather(const gputf_span *spans, uint64_t count, void *dst, int sms, cudaStream_t s);

/* Batched transcoding (batch.cu). */
struct BatchDir {
    uint64_t count;               /* strings */
    uint64_t units;               /* input code units */
    const void *in;
    const uint64_t *in_off;
    void *out;
    const uint64_t *out_off;
    DevResult *res;
    uint64_t tiles;               /* filled in by launch_batch */
    unsigned long long *status;   /* filled in by launch_batch */
    unsigned long long *errw;     /* filled in by launch_batch */
};
int batch_config_count();
uint64_t batch_min_tile_units();
cudaError_t launch_batch(int cfg, const BatchDir &d8, const BatchDir &d16, void *ws, uint64_t ws_nwords,
                         cudaStream_t s);

}  // namespace gputf

#endif
