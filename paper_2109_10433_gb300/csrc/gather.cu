/*
 * gputf_gather: copy many device byte spans into one buffer in one launch.
 *
 * A served batch takes its requests' inputs from wherever they live on the
 * device and lays them back to back, so that one batched call (CSR offsets)
 * can transcode them.  One cudaMemcpyAsync per request would cost a device
 * operation each, which dominates for small requests; this kernel moves all
 * of them at once.
 *
 * Each block copies one span at a time (grid-stride over spans).  Stores
 * are 16-byte aligned vectors; the source is read as 16-byte vectors when it
 * is aligned the same way, otherwise as five aligned 32-bit words per vector
 * joined by funnel shifts (every word read holds at least one byte of the
 * span, so no read leaves the span's own aligned words).  The bytes before
 * the first aligned vector of the destination and after the last one are
 * copied singly.
 */
#include <cstdint>

#include <cuda_runtime.h>

#include "gputf.h"
#include "kernels.h"

namespace {

__device__ __forceinline__ void copy_span(const uint8_t *__restrict__ s, uint8_t *__restrict__ d, uint64_t n)
{
    const uint64_t mis = (uint64_t)(-(intptr_t)d) & 15;
    const uint64_t head = mis < n ? mis : n;
    for (uint64_t b = threadIdx.x; b < head; b += blockDim.x) d[b] = s[b];
    const uint64_t nvec = (n - head) / 16;
    const uint8_t *sv = s + head;
    uint4 *dv = reinterpret_cast<uint4 *>(d + head);
    const unsigned sh = (unsigned)((uintptr_t)sv & 3) * 8;
    if (((uintptr_t)sv & 15) == 0) {
        const uint4 *src = reinterpret_cast<const uint4 *>(sv);
        for (uint64_t v = threadIdx.x; v < nvec; v += blockDim.x) dv[v] = __ldg(src + v);
    } else if (sh == 0) {
        const uint32_t *src = reinterpret_cast<const uint32_t *>(sv);
        for (uint64_t v = threadIdx.x; v < nvec; v += blockDim.x) {
            const uint32_t *w = src + 4 * v;
            dv[v] = make_uint4(__ldg(w), __ldg(w + 1), __ldg(w + 2), __ldg(w + 3));
        }
    } else {
        const uint32_t *src = reinterpret_cast<const uint32_t *>((uintptr_t)sv & ~(uintptr_t)3);
        for (uint64_t v = threadIdx.x; v < nvec; v += blockDim.x) {
            const uint32_t *w = src + 4 * v;
            const uint32_t w0 = __ldg(w), w1 = __ldg(w + 1), w2 = __ldg(w + 2), w3 = __ldg(w + 3),
                           w4 = __ldg(w + 4);
            dv[v] = make_uint4(__funnelshift_r(w0, w1, sh), __funnelshift_r(w1, w2, sh),
                               __funnelshift_r(w2, w3, sh), __funnelshift_r(w3, w4, sh));
        }
    }
    for (uint64_t b = head + 16 * nvec + threadIdx.x; b < n; b += blockDim.x) d[b] = s[b];
}

__global__ void __launch_bounds__(256) gather_kernel(const gputf_span *__restrict__ spans, uint64_t count,
                                                     uint8_t *__restrict__ dst)
{
    for (uint64_t i = blockIdx.x; i < count; i += gridDim.x) {
        const gputf_span sp = spans[i];
        copy_span(static_cast<const uint8_t *>(sp.src), dst + sp.dst_offset, sp.bytes);
    }
}

}  // namespace

namespace gputf {
cudaError_t launch_gather(const gputf_span *spans, uint64_t count, void *dst, int sms, cudaStream_t s)
{
    const uint64_t cap = (uint64_t)sms * 8;
    const unsigned grid = (unsigned)(count < cap ? count : cap);
    gather_kernel<<<grid, 256, 0, s>>>(spans, count, static_cast<uint8_t *>(dst));
    return cudaGetLastError();
}
}  // namespace gputf
