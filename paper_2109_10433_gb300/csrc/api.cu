/*
 * C-ABI entry points of libgputf (declared in include/gputf.h): argument
 * checks, workspace sizing, device checks and kernel launches.  No entry
 * point allocates device memory; the host forms keep a small per-device pool
 * (streams, events, 1.5 KB of mapped pinned host memory) for the process.
 */
#include <cstdint>
#include <cstring>
#include <mutex>

#include <cuda_runtime.h>

#include "gputf.h"
#include "common.cuh"
#include "kernels.h"

namespace {

thread_local int g_last_cuda_error = 0;

struct DeviceInfo {
    bool known = false;
    bool supported = false;
    int sms = 0;
};

constexpr int MAX_DEVICES = 64;
DeviceInfo g_devices[MAX_DEVICES];
std::mutex g_devices_mutex;

gputf_status cuda_status(cudaError_t e)
{
    if (e == cudaSuccess) return GPUTF_STATUS_OK;
    g_last_cuda_error = (int)e;
    return GPUTF_STATUS_CUDA_ERROR;
}

/* The current device, checked to be an sm_103 part. */
gputf_status current_device(int *sms)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e);
    if (dev < 0 || dev >= MAX_DEVICES) return GPUTF_STATUS_UNSUPPORTED_DEVICE;
    std::lock_guard<std::mutex> lock(g_devices_mutex);
    DeviceInfo &d = g_devices[dev];
    if (!d.known) {
        int major = 0, minor = 0, count = 0;
        if ((e = cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev)) != cudaSuccess ||
            (e = cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev)) != cudaSuccess ||
            (e = cudaDeviceGetAttribute(&count, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
            return cuda_status(e);
        d.supported = (major == 10 && minor == 3);
        d.sms = count;
        d.known = true;
    }
    if (!d.supported) return GPUTF_STATUS_UNSUPPORTED_DEVICE;
    *sms = d.sms;
    return GPUTF_STATUS_OK;
}

bool aligned(const void *p, uintptr_t a) { return ((uintptr_t)p & (a - 1)) == 0; }

/* Checks shared by all calls; *status_words = tile-status capacity. */
gputf_status check_common(const void *in, size_t n, void *ws, size_t ws_bytes, const void *res,
                          uintptr_t in_align, uint64_t *status_words)
{
    if ((n > 0 && in == nullptr) || ws == nullptr || res == nullptr) return GPUTF_STATUS_INVALID_ARGUMENT;
    if (!aligned(in, in_align) || !aligned(ws, 16) || !aligned(res, 8)) return GPUTF_STATUS_INVALID_ARGUMENT;
    if ((uint64_t)n > GPUTF_MAX_UNITS) return GPUTF_STATUS_INPUT_TOO_LARGE;
    if (ws_bytes < gputf::HEADER_BYTES) return GPUTF_STATUS_WORKSPACE_TOO_SMALL;
    *status_words = (ws_bytes - gputf::HEADER_BYTES) / 8;
    return GPUTF_STATUS_OK;
}

__global__ void workspace_header_init(gputf::WsHeader *h)
{
    h->err_pos = gputf::NONE;
    h->cap_pos = gputf::NONE;
    h->epoch = 1;
}

}  // namespace

namespace gputf {
gputf_status status_of(cudaError_t e) { return cuda_status(e); }

cudaError_t launch_workspace_init(void *ws, uint64_t bytes, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(ws, 0, bytes, s);
    if (e != cudaSuccess) return e;
    workspace_header_init<<<1, 1, 0, s>>>(static_cast<WsHeader *>(ws));
    return cudaGetLastError();
}
}  // namespace gputf

namespace {
gputf_status utf8_to_utf16_call(const uint8_t *in, size_t n_bytes, uint16_t *out, size_t out_cap, void *ws,
                                size_t ws_bytes, gputf_result *res, bool validate, bool big_endian,
                                bool chained, cudaStream_t stream)
{
    uint64_t words;
    gputf_status st = check_common(in, n_bytes, ws, ws_bytes, res, 1, &words);
    if (st != GPUTF_STATUS_OK) return st;
    if ((out_cap > 0 && out == nullptr) || !aligned(out, 2)) return GPUTF_STATUS_INVALID_ARGUMENT;
    if (gputf::utf8_to_utf16_tiles(in, n_bytes) > words) return GPUTF_STATUS_WORKSPACE_TOO_SMALL;
    int sms;
    if ((st = current_device(&sms)) != GPUTF_STATUS_OK) return st;
    return cuda_status(gputf::launch_utf8_to_utf16(in, n_bytes, out, out_cap, ws, words,
                                                   reinterpret_cast<gputf::DevResult *>(res), sms, validate,
                                                   big_endian, chained, stream));
}

gputf_status utf16_to_utf8_call(const uint16_t *in, size_t n_units, uint8_t *out, size_t out_cap, void *ws,
                                size_t ws_bytes, gputf_result *res, bool validate, bool big_endian,
                                bool chained, cudaStream_t stream)
{
    uint64_t words;
    gputf_status st = check_common(in, n_units, ws, ws_bytes, res, 2, &words);
    if (st != GPUTF_STATUS_OK) return st;
    if (out_cap > 0 && out == nullptr) return GPUTF_STATUS_INVALID_ARGUMENT;
    if (gputf::utf16_to_utf8_tiles(in, n_units) > words) return GPUTF_STATUS_WORKSPACE_TOO_SMALL;
    int sms;
    if ((st = current_device(&sms)) != GPUTF_STATUS_OK) return st;
    return cuda_status(gputf::launch_utf16_to_utf8(in, n_units, out, out_cap, ws, words,
                                                   reinterpret_cast<gputf::DevResult *>(res), sms, validate,
                                                   big_endian, chained, stream));
}
}  // namespace

extern "C" {

size_t gputf_workspace_bytes(size_t max_units)
{
    /* one status word per tile of at least 1024 units, plus the header */
    uint64_t tiles = ((uint64_t)max_units + 16) / 1024 + 2;
    return gputf::HEADER_BYTES + 8 * tiles;
}

gputf_status gputf_workspace_init(void *ws, size_t ws_bytes, cudaStream_t stream)
{
    if (ws == nullptr || !aligned(ws, 16) || ws_bytes < gputf::HEADER_BYTES)
        return GPUTF_STATUS_INVALID_ARGUMENT;
    int sms;
    gputf_status st = current_device(&sms);
    if (st != GPUTF_STATUS_OK) return st;
    return cuda_status(gputf::launch_workspace_init(ws, ws_bytes, stream));
}


gputf_status gputf_utf8_to_utf16(const uint8_t *in, size_t n_bytes, uint16_t *out, size_t out_cap,
                                 void *ws, size_t ws_bytes, gputf_result *res, cudaStream_t stream)
{
    return utf8_to_utf16_call(in, n_bytes, out, out_cap, ws, ws_bytes, res, true, false, false, stream);
}

gputf_status gputf_utf16_to_utf8(const uint16_t *in, size_t n_units, uint8_t *out, size_t out_cap,
                                 void *ws, size_t ws_bytes, gputf_result *res, cudaStream_t stream)
{
    return utf16_to_utf8_call(in, n_units, out, out_cap, ws, ws_bytes, res, true, false, false, stream);
}

gputf_status gputf_utf8_to_utf16_unchecked(const uint8_t *in, size_t n_bytes, uint16_t *out, size_t out_cap,
                                           void *ws, size_t ws_bytes, gputf_result *res, cudaStream_t stream)
{
    return utf8_to_utf16_call(in, n_bytes, out, out_cap, ws, ws_bytes, res, false, false, false, stream);
}

gputf_status gputf_utf16_to_utf8_unchecked(const uint16_t *in, size_t n_units, uint8_t *out, size_t out_cap,
                                           void *ws, size_t ws_bytes, gputf_result *res, cudaStream_t stream)
{
    return utf16_to_utf8_call(in, n_units, out, out_cap, ws, ws_bytes, res, false, false, false, stream);
}

gputf_status gputf_validate_utf8(const uint8_t *in, size_t n_bytes, void *ws, size_t ws_bytes,
                                 gputf_result *res, cudaStream_t stream)
{
    uint64_t words;
    gputf_status st = check_common(in, n_bytes, ws, ws_bytes, res, 1, &words);
    if (st != GPUTF_STATUS_OK) return st;
    int sms;
    if ((st = current_device(&sms)) != GPUTF_STATUS_OK) return st;
    return cuda_status(gputf::launch_validate_utf8(in, n_bytes, ws,
                                                   reinterpret_cast<gputf::DevResult *>(res), sms, stream));
}

static gputf_status validate_utf16_call(const uint16_t *in, size_t n_units, void *ws, size_t ws_bytes,
                                       gputf_result *res, bool big_endian, cudaStream_t stream)
{
    uint64_t words;
    gputf_status st = check_common(in, n_units, ws, ws_bytes, res, 2, &words);
    if (st != GPUTF_STATUS_OK) return st;
    int sms;
    if ((st = current_device(&sms)) != GPUTF_STATUS_OK) return st;
    return cuda_status(gputf::launch_validate_utf16(in, n_units, ws, reinterpret_cast<gputf::DevResult *>(res),
                                                    sms, big_endian, stream));
}

gputf_status gputf_validate_utf16(const uint16_t *in, size_t n_units, void *ws, size_t ws_bytes,
                                  gputf_result *res, cudaStream_t stream)
{
    return validate_utf16_call(in, n_units, ws, ws_bytes, res, false, stream);
}

gputf_status gputf_utf16_length_from_utf8(const uint8_t *in, size_t n_bytes, void *ws,
                                          size_t ws_bytes, uint64_t *len, cudaStream_t stream)
{
    uint64_t words;
    gputf_status st = check_common(in, n_bytes, ws, ws_bytes, len, 1, &words);
    if (st != GPUTF_STATUS_OK) return st;
    int sms;
    if ((st = current_device(&sms)) != GPUTF_STATUS_OK) return st;
    return cuda_status(gputf::launch_utf16_length_from_utf8(
        in, n_bytes, ws, reinterpret_cast<unsigned long long *>(len), sms, stream));
}

static gputf_status utf8_length_from_utf16_call(const uint16_t *in, size_t n_units, void *ws, size_t ws_bytes,
                                                uint64_t *len, bool big_endian, cudaStream_t stream)
{
    uint64_t words;
    gputf_status st = check_common(in, n_units, ws, ws_bytes, len, 2, &words);
    if (st != GPUTF_STATUS_OK) return st;
    int sms;
    if ((st = current_device(&sms)) != GPUTF_STATUS_OK) return st;
    return cuda_status(gputf::launch_utf8_length_from_utf16(
        in, n_units, ws, reinterpret_cast<unsigned long long *>(len), sms, big_endian, stream));
}

gputf_status gputf_utf8_length_from_utf16(const uint16_t *in, size_t n_units, void *ws,
                                          size_t ws_bytes, uint64_t *len, cudaStream_t stream)
{
    return utf8_length_from_utf16_call(in, n_units, ws, ws_bytes, len, false, stream);
}

gputf_status gputf_utf16be_to_utf8(const uint16_t *in, size_t n_units, uint8_t *out, size_t out_cap, void *ws,
                                   size_t ws_bytes, gputf_result *res, cudaStream_t stream)
{
    return utf16_to_utf8_call(in, n_units, out, out_cap, ws, ws_bytes, res, true, true, false, stream);
}

gputf_status gputf_utf8_to_utf16be(const uint8_t *in, size_t n_bytes, uint16_t *out, size_t out_cap, void *ws,
                                   size_t ws_bytes, gputf_result *res, cudaStream_t stream)
{
    return utf8_to_utf16_call(in, n_bytes, out, out_cap, ws, ws_bytes, res, true, true, false, stream);
}

gputf_status gputf_validate_utf16be(const uint16_t *in, size_t n_units, void *ws, size_t ws_bytes,
                                    gputf_result *res, cudaStream_t stream)
{
    return validate_utf16_call(in, n_units, ws, ws_bytes, res, true, stream);
}

gputf_status gputf_utf8_length_from_utf16be(const uint16_t *in, size_t n_units, void *ws, size_t ws_bytes,
                                            uint64_t *len, cudaStream_t stream)
{
    return utf8_length_from_utf16_call(in, n_units, ws, ws_bytes, len, true, stream);
}

size_t gputf_utf8_chunk_end(const uint8_t *in, size_t n, size_t at)
{
    if (in == nullptr || at >= n) return n;
    for (size_t k = 0; k < 4 && k <= at; k++)
        if ((in[at - k] & 0xC0) != 0x80) return at - k;
    return at;
}

size_t gputf_utf16_chunk_end(const uint16_t *in, size_t n, size_t at)
{
    if (in == nullptr || at >= n) return n;
    return (at > 0 && (in[at - 1] & 0xFC00) == 0xD800) ? at - 1 : at;
}

}  // extern "C"

namespace {

constexpr size_t HOST_MAX_CHUNKS = 64;

/* Per device, kept for the process: the host forms' two copy streams, the
 * events that order their chunks, and mapped pinned host memory that the
 * chunks' kernels write their results to (so the host reads a result without
 * a device -> host copy, which would queue behind the output copies).  The
 * lock makes host-form calls on one device take turns. */
struct HostPool {
    std::mutex m;
    bool ready = false;
    cudaStream_t in = nullptr, out = nullptr;
    cudaEvent_t start = nullptr, arrived[HOST_MAX_CHUNKS] = {}, finished[HOST_MAX_CHUNKS] = {};
    gputf::DevResult *res_h = nullptr, *res_d = nullptr;
};
HostPool g_host_pools[MAX_DEVICES];

cudaError_t host_pool_ready(HostPool &p)
{
    if (p.ready) return cudaSuccess;
    cudaError_t e;
    if ((e = cudaStreamCreateWithFlags(&p.in, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&p.out, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&p.start, cudaEventDisableTiming)) != cudaSuccess)
        return e;
    for (size_t k = 0; k < HOST_MAX_CHUNKS; k++)
        if ((e = cudaEventCreateWithFlags(&p.arrived[k], cudaEventDisableTiming)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&p.finished[k], cudaEventDisableTiming)) != cudaSuccess)
            return e;
    void *h = nullptr;
    if ((e = cudaHostAlloc(&h, HOST_MAX_CHUNKS * sizeof(gputf::DevResult), cudaHostAllocMapped | cudaHostAllocPortable)) !=
        cudaSuccess)
        return e;
    void *d = nullptr;
    if ((e = cudaHostGetDevicePointer(&d, h, 0)) != cudaSuccess) {
        cudaFreeHost(h);
        return e;
    }
    p.res_h = static_cast<gputf::DevResult *>(h);
    p.res_d = static_cast<gputf::DevResult *>(d);
    p.ready = true;
    return cudaSuccess;
}

/* Waits, on every return path, for the work a host-form call queued on the
 * pool's streams and the caller's stream (it reads and writes the caller's
 * buffers). */
struct HostDrain {
    cudaStream_t a, b, c;
    ~HostDrain()
    {
        cudaStreamSynchronize(a);
        cudaStreamSynchronize(b);
        cudaStreamSynchronize(c);
    }
};

/*
 * The host forms.  The input is cut into chunks at points where the single
 * call's results do not depend on what lies beyond (gputf_*_chunk_end): the
 * first ones chunk/8, chunk/4 and chunk/2 units long, so that output starts
 * to come back early, then `chunk`.  All host -> device copies go out at once
 * on one stream.  All chunks are launched at once on the caller's stream,
 * each after its input has arrived, chained: it writes into d_out after the
 * output units of the chunks before it, which the workspace header carries
 * from chunk to chunk on the device, within the capacity left.  Each writes
 * its result to the pool's mapped pinned memory; as each finishes, the host
 * reads its `written` and copies those units back to h_out on a third stream
 * while later chunks run.  The first chunk that reports an error or a full
 * output ends the result (the chunks after it still run, writing beyond it in
 * d_out, as the single call may), its position moved to the whole input's.
 * So h_out, d_out and the result are the single call's.
 */
template <typename TIn, typename TOut, typename Call, typename Cut>
gputf_status host_form(const TIn *h_in, size_t n, TOut *h_out, size_t out_cap, TIn *d_in, TOut *d_out,
                       void *ws, size_t ws_bytes, gputf_result *d_res, gputf_result *h_res, cudaStream_t stream,
                       size_t chunk, Call call, Cut cut)
{
    if ((n > 0 && (h_in == nullptr || d_in == nullptr)) || h_res == nullptr || d_res == nullptr ||
        (out_cap > 0 && (h_out == nullptr || d_out == nullptr)) || ws == nullptr || !aligned(ws, 16))
        return GPUTF_STATUS_INVALID_ARGUMENT;
    if (ws_bytes < gputf::HEADER_BYTES) return GPUTF_STATUS_WORKSPACE_TOO_SMALL;
    if (chunk < 64) chunk = 64;
    if (n / chunk >= HOST_MAX_CHUNKS - 4) chunk = n / (HOST_MAX_CHUNKS - 5);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e);
    if (dev < 0 || dev >= MAX_DEVICES) return GPUTF_STATUS_UNSUPPORTED_DEVICE;
    HostPool &p = g_host_pools[dev];
    std::lock_guard<std::mutex> lock(p.m);
    if ((e = host_pool_ready(p)) != cudaSuccess) return cuda_status(e);
    HostDrain drain{p.in, p.out, stream};
    if ((e = cudaEventRecord(p.start, stream)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(p.in, p.start, 0)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(p.out, p.start, 0)) != cudaSuccess)
        return cuda_status(e);

    /* chunk k is [a[k], a[k + 1]) */
    size_t a[HOST_MAX_CHUNKS + 1];
    size_t chunks = 0, step = chunk / 8 > 64 ? chunk / 8 : 64;
    a[0] = 0;
    while (a[chunks] < n || chunks == 0) {
        const size_t next = chunks + 1 == HOST_MAX_CHUNKS ? n : cut(h_in, n, a[chunks] + step);
        a[++chunks] = next;
        step = 2 * step < chunk ? 2 * step : chunk;
        if (next >= n) break;
    }
    for (size_t k = 0; k < chunks; k++) {
        const size_t len = a[k + 1] - a[k];
        if (len && (e = cudaMemcpyAsync(d_in + a[k], h_in + a[k], len * sizeof(TIn), cudaMemcpyHostToDevice,
                                        p.in)) != cudaSuccess)
            return cuda_status(e);
        if ((e = cudaEventRecord(p.arrived[k], p.in)) != cudaSuccess) return cuda_status(e);
    }
    gputf::WsHeader *hdr = static_cast<gputf::WsHeader *>(ws);
    if ((e = cudaMemsetAsync(&hdr->out_base, 0, sizeof hdr->out_base, stream)) != cudaSuccess)
        return cuda_status(e);
    for (size_t k = 0; k < chunks; k++) {
        if ((e = cudaStreamWaitEvent(stream, p.arrived[k], 0)) != cudaSuccess) return cuda_status(e);
        const gputf_status st = call(d_in + a[k], a[k + 1] - a[k], d_out, out_cap, ws, ws_bytes,
                                     reinterpret_cast<gputf_result *>(p.res_d + k), stream);
        if (st != GPUTF_STATUS_OK) return st;
        if ((e = cudaEventRecord(p.finished[k], stream)) != cudaSuccess) return cuda_status(e);
    }

    gputf_result total = {GPUTF_E_OK, 0, (uint64_t)n, 0};
    uint64_t done = 0;   /* output units of the chunks so far */
    for (size_t k = 0; k < chunks; k++) {
        if ((e = cudaEventSynchronize(p.finished[k])) != cudaSuccess) return cuda_status(e);
        const volatile gputf::DevResult *vr = p.res_h + k;
        const int32_t error = vr->error;
        const uint64_t position = vr->position, written = vr->written;
        const uint64_t w = written < out_cap - done ? written : out_cap - done;
        if (w && (e = cudaMemcpyAsync(h_out + done, d_out + done, w * sizeof(TOut), cudaMemcpyDeviceToHost,
                                      p.out)) != cudaSuccess)
            return cuda_status(e);
        done += w;
        if (error != GPUTF_E_OK) {
            total.error = error;
            total.position = error == GPUTF_E_TIMEOUT ? 0 : a[k] + position;
            total.written = error == GPUTF_E_TIMEOUT ? 0 : done;
            break;
        }
        total.written = done;
    }
    if ((e = cudaStreamSynchronize(p.out)) != cudaSuccess || (e = cudaStreamSynchronize(stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(p.in)) != cudaSuccess)
        return cuda_status(e);
    *h_res = total;
    /* the device result as the single call leaves it */
    if ((e = cudaMemcpyAsync(d_res, h_res, sizeof total, cudaMemcpyHostToDevice, stream)) != cudaSuccess)
        return cuda_status(e);
    return cuda_status(cudaStreamSynchronize(stream));
}

constexpr size_t HOST_CHUNK_BYTES = (size_t)32 << 20;   /* input bytes per chunk of the host forms */

}  // namespace

extern "C" {

gputf_status gputf_utf8_to_utf16_host_chunked(const uint8_t *h_in, size_t n_bytes, uint16_t *h_out,
                                              size_t out_cap, uint8_t *d_in, uint16_t *d_out, void *ws,
                                              size_t ws_bytes, gputf_result *d_res, gputf_result *h_res,
                                              cudaStream_t stream, size_t chunk_bytes)
{
    auto call = [](const uint8_t *in, size_t n, uint16_t *out, size_t cap, void *w, size_t wb, gputf_result *r,
                   cudaStream_t s) { return utf8_to_utf16_call(in, n, out, cap, w, wb, r, true, false, true, s); };
    return host_form(h_in, n_bytes, h_out, out_cap, d_in, d_out, ws, ws_bytes, d_res, h_res, stream, chunk_bytes,
                     call, gputf_utf8_chunk_end);
}

gputf_status gputf_utf16_to_utf8_host_chunked(const uint16_t *h_in, size_t n_units, uint8_t *h_out,
                                              size_t out_cap, uint16_t *d_in, uint8_t *d_out, void *ws,
                                              size_t ws_bytes, gputf_result *d_res, gputf_result *h_res,
                                              cudaStream_t stream, size_t chunk_units)
{
    auto call = [](const uint16_t *in, size_t n, uint8_t *out, size_t cap, void *w, size_t wb, gputf_result *r,
                   cudaStream_t s) { return utf16_to_utf8_call(in, n, out, cap, w, wb, r, true, false, true, s); };
    return host_form(h_in, n_units, h_out, out_cap, d_in, d_out, ws, ws_bytes, d_res, h_res, stream, chunk_units,
                     call, gputf_utf16_chunk_end);
}

gputf_status gputf_utf8_to_utf16_host(const uint8_t *h_in, size_t n_bytes, uint16_t *h_out,
                                      size_t out_cap, uint8_t *d_in, uint16_t *d_out, void *ws,
                                      size_t ws_bytes, gputf_result *d_res, gputf_result *h_res,
                                      cudaStream_t stream)
{
    return gputf_utf8_to_utf16_host_chunked(h_in, n_bytes, h_out, out_cap, d_in, d_out, ws, ws_bytes, d_res,
                                            h_res, stream, HOST_CHUNK_BYTES);
}

gputf_status gputf_utf16_to_utf8_host(const uint16_t *h_in, size_t n_units, uint8_t *h_out,
                                      size_t out_cap, uint16_t *d_in, uint8_t *d_out, void *ws,
                                      size_t ws_bytes, gputf_result *d_res, gputf_result *h_res,
                                      cudaStream_t stream)
{
    return gputf_utf16_to_utf8_host_chunked(h_in, n_units, h_out, out_cap, d_in, d_out, ws, ws_bytes, d_res,
                                            h_res, stream, HOST_CHUNK_BYTES / 2);
}

size_t gputf_batch_workspace_bytes(uint64_t units8, uint64_t count8, uint64_t units16, uint64_t count16)
{
    const uint64_t t = gputf::batch_min_tile_units();
    const uint64_t tiles = (units8 + t - 1) / t + 1 + (units16 + t - 1) / t + 1;
    return gputf::HEADER_BYTES + 8 * (tiles + count8 + count16);
}

int gputf_batch_config_count(void) { return gputf::batch_config_count(); }

gputf_status gputf_batch_transcode(const gputf_batch *b8, const gputf_batch *b16, int config, void *ws,
                                   size_t ws_bytes, cudaStream_t stream)
{
    gputf::BatchDir d[2] = {};
    const gputf_batch *b[2] = {b8, b16};
    for (int k = 0; k < 2; k++) {
        if (b[k] == nullptr || b[k]->count == 0) continue;
        const gputf_batch &x = *b[k];
        if (x.in_offsets == nullptr || (x.out != nullptr && x.out_offsets == nullptr) || x.results == nullptr ||
            (x.units > 0 && x.in == nullptr) || !aligned(x.results, 8) || !aligned(x.in_offsets, 8) ||
            !aligned(x.out_offsets, 8) || (k == 1 && !aligned(x.in, 2)) || (k == 0 && !aligned(x.out, 2)))
            return GPUTF_STATUS_INVALID_ARGUMENT;
        if (x.units > GPUTF_MAX_UNITS) return GPUTF_STATUS_INPUT_TOO_LARGE;
        d[k].count = x.count;
        d[k].units = x.units;
        d[k].in = x.in;
        d[k].in_off = x.in_offsets;
        d[k].out = x.out;
        d[k].out_off = x.out != nullptr ? x.out_offsets : nullptr;
        d[k].res = reinterpret_cast<gputf::DevResult *>(x.results);
    }
    if (config < 0) config = 0;
    if (config >= gputf::batch_config_count() || ws == nullptr || !aligned(ws, 16))
        return GPUTF_STATUS_INVALID_ARGUMENT;
    if (ws_bytes < gputf_batch_workspace_bytes(d[0].units, d[0].count, d[1].units, d[1].count))
        return GPUTF_STATUS_WORKSPACE_TOO_SMALL;
    int sms;
    gputf_status st = current_device(&sms);
    if (st != GPUTF_STATUS_OK) return st;
    return cuda_status(gputf::launch_batch(config, d[0], d[1], ws, (ws_bytes - gputf::HEADER_BYTES) / 8, stream));
}

gputf_status gputf_gather(const gputf_span *spans, uint64_t count, void *dst, cudaStream_t stream)
{
    if (count == 0) return GPUTF_STATUS_OK;
    if (spans == nullptr || dst == nullptr || !aligned(spans, 8)) return GPUTF_STATUS_INVALID_ARGUMENT;
    int sms;
    gputf_status st = current_device(&sms);
    if (st != GPUTF_STATUS_OK) return st;
    return cuda_status(gputf::launch_gather(spans, count, dst, sms, stream));
}

const char *gputf_error_name(int32_t error)
{
    static const char *names[] = {"OK",        "HEADER_BITS", "TOO_SHORT",        "TOO_LONG",
                                  "OVERLONG",  "TOO_LARGE",   "SURROGATE",        "OUTPUT_TOO_SMALL",
                                  "TIMEOUT",   "INTERNAL"};
    return (error >= 0 && error <= 9) ? names[error] : "UNKNOWN";
}

const char *gputf_status_name(gputf_status status)
{
    switch (status) {
    case GPUTF_STATUS_OK: return "OK";
    case GPUTF_STATUS_INVALID_ARGUMENT: return "INVALID_ARGUMENT";
    case GPUTF_STATUS_WORKSPACE_TOO_SMALL: return "WORKSPACE_TOO_SMALL";
    case GPUTF_STATUS_INPUT_TOO_LARGE: return "INPUT_TOO_LARGE";
    case GPUTF_STATUS_CUDA_ERROR: return "CUDA_ERROR";
    case GPUTF_STATUS_UNSUPPORTED_DEVICE: return "UNSUPPORTED_DEVICE";
    }
    return "UNKNOWN";
}

int gputf_last_cuda_error(void) { return g_last_cuda_error; }

int gputf_version(void) { return 100; }

}  // extern "C"
