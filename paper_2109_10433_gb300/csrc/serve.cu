/*
 * Served batches: the host side of a request loop's launch, in one call.
 *
 * A batch of requests is planned in two passes over the request array (no
 * allocation): the first counts the requests and input units of each group
 * and the gather spans; the second assigns every request its arena ranges
 * and result row and writes the metadata (gather spans, CSR offsets) into
 * the slot's pinned staging buffer.  The launch then enqueues, on one
 * stream, the metadata copy, the gather, one batched launch for the small
 * transcode requests of both directions, one for the small validate
 * requests, the single-buffer calls of the large requests (run in place on
 * their own inputs), and the copy of the results to host.
 *
 * Groups of small requests: 0 = UTF-8 transcode, 1 = UTF-8 validate,
 * 2 = UTF-16 transcode, 3 = UTF-16 validate (index = 2 * direction + op).
 * Arena layout: UTF-8 inputs of groups 0 and 1 back to back; from the next
 * 256-byte boundary the UTF-16 inputs of groups 2 and 3; then, each from a
 * 256-byte boundary, the UTF-16 outputs of group 0 (n units per request),
 * the UTF-8 outputs of group 2 (3n bytes per request), and one output region
 * per large transcode request.  Result rows: groups 0..3 in order, then the
 * large requests, each in the order given.
 * Metadata (64-bit words): the gather spans (3 words each), then the input
 * offsets of groups 0..3 (count + 1 each, in units) and the output offsets
 * of groups 0 and 2 (count + 1 each, in output units).
 */
#include <cstdint>
#include <cstring>

#include <cuda_runtime.h>

#include "gputf.h"
#include "kernels.h"

namespace {

constexpr uint64_t ALIGN = 256;
constexpr uint64_t SPAN = 64 << 10;   /* gather spans are at most this many bytes */
constexpr uint64_t NONE64 = ~0ull;

uint64_t up(uint64_t x) { return (x + ALIGN - 1) / ALIGN * ALIGN; }

struct Layout {
    uint64_t cnt[4], units[4];
    uint64_t nbig, nspans, max_big_units;
    uint64_t in_base[4], out_base[4];   /* out_base used for groups 0 and 2 */
    uint64_t big_base;
    uint64_t row_base[5];
    uint64_t off_word[6];               /* in_off of groups 0..3, out_off of groups 0 and 2 */
    uint64_t meta_words, arena_bytes;
};

uint64_t unit_bytes(const gputf_request &r) { return r.direction ? 2 : 1; }

uint64_t out_bytes(const gputf_request &r)
{
    if (r.op) return 0;
    return r.direction ? 3 * r.units : 2 * r.units;
}

uint64_t pieces(uint64_t bytes) { return (bytes + SPAN - 1) / SPAN; }

gputf_status count_pass(const gputf_request *reqs, uint64_t count, uint64_t big_units, Layout &L)
{
    std::memset(&L, 0, sizeof L);
    if (count > 0 && reqs == nullptr) return GPUTF_STATUS_INVALID_ARGUMENT;
    uint64_t big_out = 0;
    for (uint64_t i = 0; i < count; i++) {
        const gputf_request &r = reqs[i];
        if (r.direction > 1 || r.op > 1 || (r.units > 0 && r.in == nullptr) ||
            (r.direction == 1 && ((uintptr_t)r.in & 1)))
            return GPUTF_STATUS_INVALID_ARGUMENT;
        if (r.units > GPUTF_MAX_UNITS) return GPUTF_STATUS_INPUT_TOO_LARGE;
        if (r.units >= big_units) {
            L.nbig++;
            if (r.units > L.max_big_units) L.max_big_units = r.units;
            big_out += up(out_bytes(r));
        } else {
            const int g = (int)(2 * r.direction + r.op);
            L.cnt[g]++;
            L.units[g] += r.units;
            L.nspans += pieces(r.units * unit_bytes(r));
        }
    }
    uint64_t pos = 0;
    L.in_base[0] = 0;
    L.in_base[1] = L.units[0];
    pos = up(L.units[0] + L.units[1]);
    L.in_base[2] = pos;
    L.in_base[3] = pos + 2 * L.units[2];
    pos += 2 * (L.units[2] + L.units[3]);
    L.out_base[0] = up(pos);
    pos = L.out_base[0] + 2 * L.units[0];
    L.out_base[2] = up(pos);
    pos = L.out_base[2] + 3 * L.units[2];
    L.big_base = up(pos);
    L.arena_bytes = L.big_base + big_out;
    L.row_base[0] = 0;
    for (int g = 0; g < 4; g++) L.row_base[g + 1] = L.row_base[g] + L.cnt[g];
    uint64_t w = 3 * L.nspans;
    for (int g = 0; g < 4; g++) {
        L.off_word[g] = w;
        w += L.cnt[g] + 1;
    }
    L.off_word[4] = w;
    w += L.cnt[0] + 1;
    L.off_word[5] = w;
    w += L.cnt[2] + 1;
    L.meta_words = w;
    return GPUTF_STATUS_OK;
}

/* Second pass: placements, and the metadata when meta != NULL. */
void fill_pass(const gputf_request *reqs, uint64_t count, uint64_t big_units, const Layout &L,
               gputf_placement *place, uint64_t *meta)
{
    uint64_t k[4] = {0, 0, 0, 0}, in_u[4] = {0, 0, 0, 0}, out_u[4] = {0, 0, 0, 0};
    uint64_t span = 0, big = 0, big_pos = L.big_base;
    for (uint64_t i = 0; i < count; i++) {
        const gputf_request &r = reqs[i];
        gputf_placement p;
        if (r.units >= big_units) {
            p.row = L.row_base[4] + big++;
            p.in_offset = NONE64;
            p.out_offset = r.op ? NONE64 : big_pos;
            big_pos += up(out_bytes(r));
        } else {
            const int g = (int)(2 * r.direction + r.op);
            const uint64_t ub = unit_bytes(r);
            p.row = L.row_base[g] + k[g];
            p.in_offset = L.in_base[g] + in_u[g] * ub;
            p.out_offset = NONE64;
            if (g == 0 || g == 2) p.out_offset = L.out_base[g] + out_u[g] * (g == 0 ? 2 : 1);
            if (meta) {
                meta[L.off_word[g] + k[g]] = in_u[g];
                if (g == 0) meta[L.off_word[4] + k[0]] = out_u[0];
                if (g == 2) meta[L.off_word[5] + k[2]] = out_u[2];
                const uint64_t bytes = r.units * ub;
                for (uint64_t a = 0; a < bytes; a += SPAN) {
                    meta[3 * span + 0] = (uint64_t)(uintptr_t)r.in + a;
                    meta[3 * span + 1] = p.in_offset + a;
                    meta[3 * span + 2] = bytes - a < SPAN ? bytes - a : SPAN;
                    span++;
                }
            }
            in_u[g] += r.units;
            if (g == 0) out_u[0] += r.units;
            if (g == 2) out_u[2] += 3 * r.units;
            k[g]++;
        }
        if (place) place[i] = p;
    }
    if (meta) {
        for (int g = 0; g < 4; g++) meta[L.off_word[g] + L.cnt[g]] = in_u[g];
        meta[L.off_word[4] + L.cnt[0]] = out_u[0];
        meta[L.off_word[5] + L.cnt[2]] = out_u[2];
    }
}

gputf_status cuda_ok(cudaError_t e) { return gputf::status_of(e); }

}  // namespace

extern "C" {

size_t gputf_serve_meta_bytes(uint64_t max_requests, uint64_t arena_bytes)
{
    /* spans: at most one per SPAN bytes of gathered input plus one per
     * request; offsets: at most max_requests + 4 and max_requests + 2 */
    return 8 * (3 * (arena_bytes / SPAN + max_requests + 1) + 2 * max_requests + 6 + 16);
}

gputf_status gputf_serve_plan(const gputf_request *reqs, uint64_t count, uint64_t big_units,
                              gputf_placement *place, uint64_t *arena_bytes, uint64_t *meta_bytes)
{
    Layout L;
    gputf_status st = count_pass(reqs, count, big_units, L);
    if (st != GPUTF_STATUS_OK) return st;
    fill_pass(reqs, count, big_units, L, place, nullptr);
    if (arena_bytes) *arena_bytes = L.arena_bytes;
    if (meta_bytes) *meta_bytes = 8 * L.meta_words;
    return GPUTF_STATUS_OK;
}

gputf_status gputf_serve_launch(const gputf_slot *slot, const gputf_request *reqs, uint64_t count,
                                uint64_t big_units, int config, gputf_placement *place, cudaStream_t stream)
{
    if (slot == nullptr || slot->arena == nullptr || slot->meta == nullptr || slot->meta_host == nullptr ||
        slot->results == nullptr || slot->ws == nullptr || ((uintptr_t)slot->arena & (ALIGN - 1)) ||
        ((uintptr_t)slot->meta & 7) || ((uintptr_t)slot->meta_host & 7) || ((uintptr_t)slot->results & 7))
        return GPUTF_STATUS_INVALID_ARGUMENT;
    Layout L;
    gputf_status st = count_pass(reqs, count, big_units, L);
    if (st != GPUTF_STATUS_OK) return st;
    if (count == 0) return GPUTF_STATUS_OK;
    if (count > slot->max_requests || L.arena_bytes > slot->arena_bytes || 8 * L.meta_words > slot->meta_bytes)
        return GPUTF_STATUS_WORKSPACE_TOO_SMALL;
    const uint64_t need_ws = gputf_batch_workspace_bytes(L.units[0], L.cnt[0], L.units[2], L.cnt[2]);
    const uint64_t need_ws_v = gputf_batch_workspace_bytes(L.units[1], L.cnt[1], L.units[3], L.cnt[3]);
    if (slot->ws_bytes < need_ws || slot->ws_bytes < need_ws_v) return GPUTF_STATUS_WORKSPACE_TOO_SMALL;
    if (L.nbig && (slot->ws1 == nullptr || slot->ws1_bytes < gputf_workspace_bytes(L.max_big_units)))
        return GPUTF_STATUS_WORKSPACE_TOO_SMALL;

    uint64_t *meta_h = static_cast<uint64_t *>(slot->meta_host);
    fill_pass(reqs, count, big_units, L, place, meta_h);
    char *arena = static_cast<char *>(slot->arena);
    const uint64_t *meta_d = static_cast<const uint64_t *>(slot->meta);

    st = cuda_ok(cudaMemcpyAsync(slot->meta, slot->meta_host, 8 * L.meta_words, cudaMemcpyHostToDevice, stream));
    if (st != GPUTF_STATUS_OK) return st;
    if (L.nspans) {
        st = gputf_gather(reinterpret_cast<const gputf_span *>(meta_d), L.nspans, arena, stream);
        if (st != GPUTF_STATUS_OK) return st;
    }
    gputf_batch b[4];
    for (int g = 0; g < 4; g++) {
        const bool writes = g == 0 || g == 2;
        b[g].count = L.cnt[g];
        b[g].units = L.units[g];
        b[g].in = arena + L.in_base[g];
        b[g].in_offsets = meta_d + L.off_word[g];
        b[g].out = writes ? arena + L.out_base[g] : nullptr;
        b[g].out_offsets = writes ? meta_d + L.off_word[g == 0 ? 4 : 5] : nullptr;
        b[g].results = slot->results + L.row_base[g];
    }
    if (L.cnt[0] || L.cnt[2]) {
        st = gputf_batch_transcode(L.cnt[0] ? &b[0] : nullptr, L.cnt[2] ? &b[2] : nullptr, config, slot->ws,
                                   slot->ws_bytes, stream);
        if (st != GPUTF_STATUS_OK) return st;
    }
    if (L.cnt[1] || L.cnt[3]) {
        st = gputf_batch_transcode(L.cnt[1] ? &b[1] : nullptr, L.cnt[3] ? &b[3] : nullptr, config, slot->ws,
                                   slot->ws_bytes, stream);
        if (st != GPUTF_STATUS_OK) return st;
    }
    uint64_t big = 0, big_pos = L.big_base;
    for (uint64_t i = 0; i < count && big < L.nbig; i++) {
        const gputf_request &r = reqs[i];
        if (r.units < big_units) continue;
        gputf_result *res = slot->results + L.row_base[4] + big++;
        if (r.op == 0) {
            void *out = arena + big_pos;
            st = r.direction == 0
                     ? gputf_utf8_to_utf16(static_cast<const uint8_t *>(r.in), r.units, static_cast<uint16_t *>(out),
                                           r.units, slot->ws1, slot->ws1_bytes, res, stream)
                     : gputf_utf16_to_utf8(static_cast<const uint16_t *>(r.in), r.units, static_cast<uint8_t *>(out),
                                           3 * r.units, slot->ws1, slot->ws1_bytes, res, stream);
            big_pos += up(out_bytes(r));
        } else {
            st = r.direction == 0
                     ? gputf_validate_utf8(static_cast<const uint8_t *>(r.in), r.units, slot->ws1, slot->ws1_bytes,
                                           res, stream)
                     : gputf_validate_utf16(static_cast<const uint16_t *>(r.in), r.units, slot->ws1,
                                            slot->ws1_bytes, res, stream);
        }
        if (st != GPUTF_STATUS_OK) return st;
    }
    if (slot->results_host)
        st = cuda_ok(cudaMemcpyAsync(slot->results_host, slot->results, count * sizeof(gputf_result),
                                     cudaMemcpyDeviceToHost, stream));
    return st;
}

}  // extern "C"
