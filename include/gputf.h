/*
 * gputf: validating UTF-8 <-> UTF-16 transcoding on NVIDIA GB300 (sm_103a).
 *
 * The problem is the one stated by Lemire & Mula, "Transcoding Billions of
 * Unicode Characters per Second with SIMD Instructions" (arXiv 2109.10433):
 * transcode input in either UTF-8 or UTF-16 to the other encoding, with
 * validation (Section 1), where validity is defined by the format rules of
 * Section 3 (UTF-8 validation rules 1-6; UTF-16 surrogate pairs) and the
 * transcoder reports how much input it consumed and how much output it
 * wrote (Algorithm 3).
 *
 * Conventions shared by every call:
 *   - Units.  Sizes and positions count code units of the encoding they refer
 *     to: bytes for UTF-8, 16-bit units for UTF-16.  UTF-16 is little-endian
 *     except in the calls named utf16be, which take big-endian units; no
 *     byte-order mark is detected or removed (U+FEFF is an ordinary
 *     character), and U+0000 is an ordinary character.
 *   - Memory.  `in`, `out`, the workspace and `res`/`len` are memory the
 *     caller owns: device memory (for example from torch.empty on a CUDA
 *     device), except that `res` and `len` may also be mapped pinned host
 *     memory.  UTF-16 pointers must be 2-byte aligned, the workspace 16-byte
 *     aligned, `res` and `len` 8-byte aligned; UTF-8 pointers need no
 *     alignment.  No call allocates memory.
 *   - Asynchrony.  Every call enqueues its work on `stream` and returns; the
 *     result is written to `res` (or `len`) by the GPU.  Read it after the
 *     stream has been synchronised.
 *   - Workspace.  Calls that write output, validate or count use a workspace
 *     of at least gputf_workspace_bytes(n) bytes, prepared once with
 *     gputf_workspace_init().  The library keeps it ready for the next call
 *     itself.  One workspace serves one call at a time: calls that share a
 *     workspace must be ordered (for example, on one stream).
 *   - Errors.  A gputf_status reports whether the call could be enqueued
 *     (bad arguments, workspace too small, CUDA launch failure).  Whether the
 *     data is valid is reported in the gputf_result.
 */
#ifndef GPUTF_H
#define GPUTF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

struct CUstream_st;
typedef struct CUstream_st *cudaStream_t;

/* Data-level outcome (gputf_result.error).  Classes 1-6 follow the UTF-8
 * validation rules of Section 3; UTF-16 input only ever reports
 * GPUTF_SURROGATE.  When several rules fail on one character the class is
 * taken in decoding order: the lead byte (TOO_LONG, HEADER_BITS), then
 * missing continuation bytes (TOO_SHORT), then OVERLONG, TOO_LARGE,
 * SURROGATE. */
typedef enum gputf_error {
    GPUTF_OK = 0,
    GPUTF_HEADER_BITS = 1,       /* rule 1: a byte 0xF8..0xFF                         */
    GPUTF_TOO_SHORT = 2,         /* rule 2: a lead without enough continuation bytes  */
    GPUTF_TOO_LONG = 3,          /* rule 3: a continuation byte without a lead        */
    GPUTF_OVERLONG = 4,          /* rule 4: a value that fits a shorter sequence      */
    GPUTF_TOO_LARGE = 5,         /* rule 5: a value above U+10FFFF                    */
    GPUTF_SURROGATE = 6,         /* rule 6 / Section 3: U+D800-DFFF, unpaired unit    */
    GPUTF_OUTPUT_TOO_SMALL = 7,  /* the next character does not fit in `out`          */
    GPUTF_TIMEOUT = 8,           /* a bounded wait between thread blocks ran out      */
    GPUTF_INTERNAL = 9           /* internal inconsistency (never expected)           */
} gputf_error;

/* Call-level status (return value). */
typedef enum gputf_status {
    GPUTF_STATUS_OK = 0,
    GPUTF_STATUS_INVALID_ARGUMENT = 1,   /* null pointer with n > 0, misaligned pointer */
    GPUTF_STATUS_WORKSPACE_TOO_SMALL = 2,
    GPUTF_STATUS_INPUT_TOO_LARGE = 3,    /* n above GPUTF_MAX_UNITS                      */
    GPUTF_STATUS_CUDA_ERROR = 4,         /* a CUDA call failed (see gputf_last_cuda_error) */
    GPUTF_STATUS_UNSUPPORTED_DEVICE = 5  /* the current device is not sm_103             */
} gputf_status;

/* Largest input, in code units, that one call accepts. */
#define GPUTF_MAX_UNITS (((uint64_t)1) << 38)

/* Result of a transcoding or validation call (written by the GPU).
 *   error    : GPUTF_OK or the class of the first failure;
 *   position : on success n; otherwise the offset, in input code units, of
 *              the start of the first character that is invalid or does not
 *              fit in the output (a stray continuation byte is its own start);
 *   written  : output code units of the valid prefix [0, position), which
 *              are exactly the transcoding of that prefix; output beyond them
 *              is unspecified but never goes past the capacity.  Validation
 *              calls write 0. */
typedef struct gputf_result {
    int32_t error;
    int32_t reserved;
    uint64_t position;
    uint64_t written;
} gputf_result;

/* Workspace bytes needed for inputs of up to `max_units` code units. */
size_t gputf_workspace_bytes(size_t max_units);

/* Prepares a workspace (device memory, `ws_bytes` long) for use; enqueued on
 * `stream`.  Needed once after allocation.  Every call leaves the workspace
 * ready for the next one, including a call that reported GPUTF_TIMEOUT (its
 * last thread block resets the header and moves the call epoch on); running
 * this again is harmless. */
gputf_status gputf_workspace_init(void *ws, size_t ws_bytes, cudaStream_t stream);

/* Validating UTF-8 -> UTF-16LE (Sections 3-4).
 *   in, n_bytes   : UTF-8 input (device), any alignment;
 *   out, out_cap  : UTF-16LE output (device), capacity in 16-bit units; n_bytes
 *                   units always suffice, gputf_utf16_length_from_utf8 gives the
 *                   exact need of valid input;
 *   res           : result (see gputf_result). */
gputf_status gputf_utf8_to_utf16(const uint8_t *in, size_t n_bytes, uint16_t *out, size_t out_cap,
                                 void *ws, size_t ws_bytes, gputf_result *res, cudaStream_t stream);

/* Validating UTF-16LE -> UTF-8 (Sections 3 and 5).
 *   in, n_units   : UTF-16LE input (device, 2-byte aligned);
 *   out, out_cap  : UTF-8 output (device), capacity in bytes; 3 * n_units
 *                   always suffice, gputf_utf8_length_from_utf16 gives the
 *                   exact need of valid input. */
gputf_status gputf_utf16_to_utf8(const uint16_t *in, size_t n_units, uint8_t *out, size_t out_cap,
                                 void *ws, size_t ws_bytes, gputf_result *res, cudaStream_t stream);

/* Transcoding without validation (the paper's non-validating transcoders,
 * Table 4): the caller vouches that the input is valid.  Same arguments,
 * workspace and capacity rules as the validating calls; on valid input the
 * result and output are identical to theirs.  On invalid input nothing is
 * checked: res->error is GPUTF_OK or GPUTF_OUTPUT_TOO_SMALL, the output is
 * unspecified, and still nothing is written past out_cap. */
gputf_status gputf_utf8_to_utf16_unchecked(const uint8_t *in, size_t n_bytes, uint16_t *out, size_t out_cap,
                                           void *ws, size_t ws_bytes, gputf_result *res, cudaStream_t stream);
gputf_status gputf_utf16_to_utf8_unchecked(const uint16_t *in, size_t n_units, uint8_t *out, size_t out_cap,
                                           void *ws, size_t ws_bytes, gputf_result *res, cudaStream_t stream);

/* Validation only (Section 3, UTF-8 rules 1-6): res->error and res->position
 * as for gputf_utf8_to_utf16, res->written = 0. */
gputf_status gputf_validate_utf8(const uint8_t *in, size_t n_bytes, void *ws, size_t ws_bytes,
                                 gputf_result *res, cudaStream_t stream);

/* Validation only (Section 3, UTF-16 surrogate pairs). */
gputf_status gputf_validate_utf16(const uint16_t *in, size_t n_units, void *ws, size_t ws_bytes,
                                  gputf_result *res, cudaStream_t stream);

/* UTF-16 length of UTF-8 input, without validation (Table 2): one unit per
 * byte that is not a continuation byte, plus one per byte >= 0xF0.  Equals
 * the transcoded length when the input is valid. */
gputf_status gputf_utf16_length_from_utf8(const uint8_t *in, size_t n_bytes, void *ws,
                                          size_t ws_bytes, uint64_t *len, cudaStream_t stream);

/* UTF-8 length of UTF-16 input, without validation (Table 2): 1, 2 or 3 bytes
 * per unit by value, 2 per surrogate unit.  Equals the transcoded length when
 * the input is valid. */
gputf_status gputf_utf8_length_from_utf16(const uint16_t *in, size_t n_units, void *ws,
                                          size_t ws_bytes, uint64_t *len, cudaStream_t stream);

/* Big-endian UTF-16 (UTF-16BE).  The paper treats UTF-16LE only (Section 3:
 * the byte order of the host); these are the same four operations on 16-bit
 * units stored most significant byte first, with the same arguments,
 * workspace, capacity and result rules as the UTF-16LE calls above.  Each
 * gives what the UTF-16LE call gives on the byte-swapped units (and, for
 * gputf_utf8_to_utf16be, writes the byte-swapped units).  `in` and `out` are
 * still 2-byte aligned arrays of 16-bit units. */
gputf_status gputf_utf16be_to_utf8(const uint16_t *in, size_t n_units, uint8_t *out, size_t out_cap,
                                   void *ws, size_t ws_bytes, gputf_result *res, cudaStream_t stream);
gputf_status gputf_utf8_to_utf16be(const uint8_t *in, size_t n_bytes, uint16_t *out, size_t out_cap,
                                   void *ws, size_t ws_bytes, gputf_result *res, cudaStream_t stream);
gputf_status gputf_validate_utf16be(const uint16_t *in, size_t n_units, void *ws, size_t ws_bytes,
                                    gputf_result *res, cudaStream_t stream);
gputf_status gputf_utf8_length_from_utf16be(const uint16_t *in, size_t n_units, void *ws,
                                            size_t ws_bytes, uint64_t *len, cudaStream_t stream);

/* Host-buffer forms of the two transcoders, for callers whose text lives in
 * host memory: copies `h_in` to the device buffer `d_in`, transcodes into
 * `d_out`, and copies the `written` output units back to `h_out`.  The
 * result goes to `h_res` and to `d_res`.  The calls are synchronous: they
 * return after the copies are done.  The device buffers are the caller's:
 * `d_in` holds the input, `d_out` out_cap units, `d_res` one gputf_result.
 * Pinned host memory makes the copies fastest.
 *
 * The input is cut into chunks at the points gputf_utf8_chunk_end /
 * gputf_utf16_chunk_end give: about 4, 8 and 16 MiB, then 32 MiB each.  All
 * host -> device copies are issued at once, and all chunks are launched at
 * once on `stream`, each after its input has arrived.  Each chunk writes its
 * output into d_out after the output of the chunks before it (the workspace
 * carries that count from chunk to chunk on the device), within the capacity
 * left.  As each chunk finishes, its output is copied back while later
 * chunks run, so the copies in both directions and the kernels overlap.  The
 * first chunk that reports an error or a full output gives the result.
 * `h_out`, `d_out` and the result are those of the single call on the whole
 * input (past the written units, d_out may hold more output, as it may after
 * the single call).  The first call on a device creates two streams, some
 * events and 1.5 KB of mapped pinned host memory for the chunks' results,
 * kept for the process; calls on one device take turns.  The calls allocate
 * no device memory.  They must not run inside a stream capture. */
gputf_status gputf_utf8_to_utf16_host(const uint8_t *h_in, size_t n_bytes, uint16_t *h_out,
                                      size_t out_cap, uint8_t *d_in, uint16_t *d_out, void *ws,
                                      size_t ws_bytes, gputf_result *d_res, gputf_result *h_res,
                                      cudaStream_t stream);
gputf_status gputf_utf16_to_utf8_host(const uint16_t *h_in, size_t n_units, uint8_t *h_out,
                                      size_t out_cap, uint16_t *d_in, uint8_t *d_out, void *ws,
                                      size_t ws_bytes, gputf_result *d_res, gputf_result *h_res,
                                      cudaStream_t stream);

/* The same with the chunk size chosen by the caller, in input code units
 * (the first three chunks an eighth, a quarter and half of it).  It is raised
 * to 64, and to n / 59 when n / chunk would reach 60 (at most 64 chunks).
 * The default forms above pass 32 MiB of input. */
gputf_status gputf_utf8_to_utf16_host_chunked(const uint8_t *h_in, size_t n_bytes, uint16_t *h_out,
                                              size_t out_cap, uint8_t *d_in, uint16_t *d_out, void *ws,
                                              size_t ws_bytes, gputf_result *d_res, gputf_result *h_res,
                                              cudaStream_t stream, size_t chunk_bytes);
gputf_status gputf_utf16_to_utf8_host_chunked(const uint16_t *h_in, size_t n_units, uint8_t *h_out,
                                              size_t out_cap, uint16_t *d_in, uint8_t *d_out, void *ws,
                                              size_t ws_bytes, gputf_result *d_res, gputf_result *h_res,
                                              cudaStream_t stream, size_t chunk_units);

/* Chunk boundaries for splitting one input into pieces transcoded by
 * separate calls.  Each function returns a position p <= at, or n when
 * at >= n.  The single call on in[0, n) gives the same result as the call
 * on in[0, p) followed, when that one succeeds, by the call on in[p, n):
 * the same output, written counts that add up, and the first error at the
 * same position, shifted by p when it lies in the second piece.
 *   UTF-8  : the last of in[at], in[at-1], in[at-2], in[at-3] that is not a
 *            continuation byte (10xxxxxx), else `at`.  A character starts
 *            there (Section 3, rule 3), or in[at] is a stray continuation
 *            byte that no character can include (at most three follow a
 *            lead).
 *   UTF-16 : at - 1 when in[at - 1] is a high surrogate (Section 3: it pairs
 *            with the unit after it, or is an error either way), else `at`.
 * Host code only: `in` is host memory, read at most 4 units before `at`. */
size_t gputf_utf8_chunk_end(const uint8_t *in, size_t n, size_t at);
size_t gputf_utf16_chunk_end(const uint16_t *in, size_t n, size_t at);

/* One direction of a batch: `count` strings stored back to back.
 *   in, in_offsets : device; string s is in[in_offsets[s] .. in_offsets[s+1])
 *                    in code units of its encoding (bytes, or 16-bit units on
 *                    a 2-byte aligned buffer); count + 1 non-decreasing
 *                    offsets starting at 0; empty strings are allowed;
 *   units          : in_offsets[count], given here so that no device read is
 *                    needed to size the launch;
 *   out, out_offsets : device; string s may write output code units
 *                    out[out_offsets[s] .. out_offsets[s+1]) (its capacity);
 *                    out == NULL validates only: nothing is written, no
 *                    capacity applies, out_offsets is ignored (may be NULL)
 *                    and each result is what gputf_validate_utf8 /
 *                    gputf_validate_utf16 gives the string (`written` 0);
 *   results        : device; count results, as gputf_result for a single
 *                    string, positions and `written` relative to the string. */
typedef struct gputf_batch {
    uint64_t count;
    uint64_t units;
    const void *in;
    const uint64_t *in_offsets;
    void *out;
    const uint64_t *out_offsets;
    gputf_result *results;
} gputf_batch;

/* Workspace bytes for a batch with the given input units and strings per
 * direction (UTF-8 -> UTF-16, then UTF-16 -> UTF-8). */
size_t gputf_batch_workspace_bytes(uint64_t units8, uint64_t count8, uint64_t units16, uint64_t count16);

/* Number of tile configurations gputf_batch_transcode accepts (0 .. n-1):
 * threads and units per thread, each either one CTA per tile or a
 * persistent grid of resident CTAs taking tiles until none is left; an
 * autotuner picks one per input mix. */
int gputf_batch_config_count(void);

/* Batched validating transcoding of many strings in one launch (the paper's
 * single-string transcoders of Sections 4-5 applied to every string; tiles
 * of the launch cross string boundaries).  Either direction may be NULL or
 * have count 0.  Each string gets exactly the result and output that the
 * single-string call would give it.  `config` selects the tile shape.
 * Enqueued on `stream`; allocates nothing, so it can be captured into a CUDA
 * graph. */
gputf_status gputf_batch_transcode(const gputf_batch *utf8_to_utf16, const gputf_batch *utf16_to_utf8,
                                   int config, void *ws, size_t ws_bytes, cudaStream_t stream);

/* A batched launch recorded into a CUDA graph, for replay. */
typedef struct gputf_graph gputf_graph;

/* Records gputf_batch_transcode(...) on `stream` (which must not be the
 * legacy default stream, nor already capturing) into a graph and
 * instantiates it; *graph receives the handle.  Replays transcode the same
 * device buffers again, with whatever they hold at replay time.  Creating the
 * graph allocates host-side graph objects; replaying does not. */
gputf_status gputf_batch_graph_create(const gputf_batch *utf8_to_utf16, const gputf_batch *utf16_to_utf8,
                                      int config, void *ws, size_t ws_bytes, cudaStream_t stream,
                                      gputf_graph **graph);
/* Enqueues one replay of the graph on `stream`. */
gputf_status gputf_graph_launch(gputf_graph *graph, cudaStream_t stream);
/* Releases the graph. */
void gputf_graph_destroy(gputf_graph *graph);

/* One span of a gather: `bytes` bytes at device address `src`, copied to
 * dst + dst_offset. */
typedef struct gputf_span {
    const void *src;
    uint64_t dst_offset;
    uint64_t bytes;
} gputf_span;

/* Copies `count` spans into the device buffer `dst` in one launch.  The
 * paper has no counterpart: this assembles many requests' inputs, wherever
 * they sit on the device, into the back-to-back layout that
 * gputf_batch_transcode reads (the served form of the batched call).
 *   spans : device array of `count` spans, 8-byte aligned; sources and
 *           destinations may have any alignment; destination ranges must
 *           not overlap each other or any source.  A block copies one span
 *           at a time, so very long spans are best split by the caller.
 * Enqueued on `stream`; allocates nothing.  INVALID_ARGUMENT for NULL
 * pointers with count > 0. */
gputf_status gputf_gather(const gputf_span *spans, uint64_t count, void *dst, cudaStream_t stream);

/* ---------------------------------------------------------------------------
 * Served batches.  The paper has no counterpart: these calls turn a set of
 * independent requests into the calls above (one gather, one batched
 * transcode launch, one batched validate launch, one single-buffer call per
 * large request), so that a request loop can hand the library a whole batch
 * at once.  Every request gets the result (and output) of the single call on
 * its input.
 * ------------------------------------------------------------------------ */

/* One request.  `in` is device memory holding `units` input code units (a
 * UTF-16 input 2-byte aligned). */
typedef struct gputf_request {
    const void *in;
    uint64_t units;
    uint32_t direction;   /* 0: UTF-8 -> UTF-16LE, 1: UTF-16LE -> UTF-8        */
    uint32_t op;          /* 0: transcode, 1: validate only                     */
} gputf_request;

/* Where a request of a planned batch goes. */
typedef struct gputf_placement {
    uint64_t row;          /* its result: results[row]                              */
    uint64_t in_offset;    /* arena byte offset of its gathered input; UINT64_MAX
                              when it runs in place (units >= big_units)             */
    uint64_t out_offset;   /* arena byte offset of its output (capacity: n UTF-16
                              units, or 3n UTF-8 bytes); UINT64_MAX when validating */
} gputf_placement;

/* The device and pinned host memory one batch slot owns, all caller-owned.
 *   arena / arena_bytes : device, 256-byte aligned; inputs gathered back to
 *                         back, then outputs;
 *   meta / meta_host / meta_bytes : device and pinned host buffers of the same
 *                         size (gputf_serve_meta_bytes), 8-byte aligned: gather
 *                         spans and CSR offsets, written to meta_host and copied;
 *   results / results_host : device and pinned host arrays of max_requests
 *                         results; the results are copied back at the end;
 *   ws, ws_bytes   : workspace of at least gputf_batch_workspace_bytes(
 *                    arena_bytes, max_requests, arena_bytes / 2, max_requests);
 *   ws1, ws1_bytes : workspace of at least gputf_workspace_bytes(u), u the
 *                    largest request run in place.
 * A slot serves one batch at a time: meta_host and results_host may be
 * touched again only once the stream has passed the batch. */
typedef struct gputf_slot {
    void *arena;
    uint64_t arena_bytes;
    void *meta;
    void *meta_host;
    uint64_t meta_bytes;
    gputf_result *results;
    gputf_result *results_host;
    uint64_t max_requests;
    void *ws;
    uint64_t ws_bytes;
    void *ws1;
    uint64_t ws1_bytes;
} gputf_slot;

/* Bytes of metadata a slot needs for up to max_requests requests whose
 * gathered inputs fill at most arena_bytes. */
size_t gputf_serve_meta_bytes(uint64_t max_requests, uint64_t arena_bytes);

/* Plans a batch without touching the GPU: requests with units >= big_units
 * run in place; the others are grouped by (direction, op) in the order
 * given.  place[i] receives request i's placement; *arena_bytes and
 * *meta_bytes the arena and metadata the batch needs.  INVALID_ARGUMENT for
 * a bad direction or op, a NULL pointer, or a misaligned UTF-16 input. */
gputf_status gputf_serve_plan(const gputf_request *reqs, uint64_t count, uint64_t big_units,
                              gputf_placement *place, uint64_t *arena_bytes, uint64_t *meta_bytes);

/* Plans (as above) and enqueues one batch on `stream`: the metadata copy,
 * the gather of the small requests' inputs (gputf_gather), the batched
 * transcode and validate launches (gputf_batch_transcode with `config`),
 * one single-buffer call per large request, and the copy of the results to
 * results_host.  WORKSPACE_TOO_SMALL when the batch needs more arena,
 * metadata, result rows or workspace than the slot has; nothing is enqueued
 * then.  Allocates nothing. */
gputf_status gputf_serve_launch(const gputf_slot *slot, const gputf_request *reqs, uint64_t count,
                                uint64_t big_units, int config, gputf_placement *place,
                                cudaStream_t stream);

/* Largest input, in 16-bit units, that gputf_utf16_to_utf8_static accepts
 * (32 Mi units, 64 MiB of UTF-16). */
#define GPUTF_STATIC_MAX_UNITS (((uint64_t)1) << 25)

/* gputf_utf16_to_utf8 for callers that cannot allocate device memory (the
 * paper has no counterpart: this is a deployment concern).  Some callers
 * must not call cudaMalloc when they run: code on a stream that is being
 * captured into a CUDA graph in a mode that forbids it, code inside a custom
 * allocator or memory-pool callback, where allocating would re-enter the
 * allocator, or a service that reserves all its memory at start-up.  This
 * entry point takes no workspace: its scratch is a fixed array inside the
 * library (about 256 KiB), which every GPU that loads the library keeps until
 * the process exits.  Arguments, results and units are as for
 * gputf_utf16_to_utf8.
 *   - Inputs longer than GPUTF_STATIC_MAX_UNITS are refused with
 *     GPUTF_STATUS_INPUT_TOO_LARGE; use gputf_utf16_to_utf8 for those.
 *   - The first call on each device sets the scratch up (it looks up the
 *     array's device address and enqueues its initialisation on `stream`);
 *     make that first call before any stream capture: made on a stream that
 *     is being captured, it returns GPUTF_STATUS_INVALID_ARGUMENT and does
 *     nothing.  The set-up is remembered per device for the life of the
 *     process, in the primary context: after cudaDeviceReset, or from
 *     another context on the same device, this call is not valid.
 *   - A call that reports GPUTF_TIMEOUT leaves the scratch ready for the
 *     next call, as for a workspace (its last thread block resets it).
 *   - All calls on a device share the one array: calls that overlap on the
 *     GPU (on different streams without ordering) race and must be avoided.
 *   - Allocates nothing: no cudaMalloc, no cudaFree, no allocating library
 *     routine. */
gputf_status gputf_utf16_to_utf8_static(const uint16_t *in, size_t n_units, uint8_t *out,
                                        size_t out_cap, gputf_result *res, cudaStream_t stream);

/* Failure detection, for tests: runs one of the kernels' bounded waits until
 * it gives up, as a call whose data never arrives would (the paper has no
 * counterpart).  which = 0: the decoupled look-back of the output offsets
 * (A3), polling the status word of a tile that never publishes; which = 1:
 * the wait on a shared-memory barrier that a tile copy completes (A1), with
 * no copy issued.  `polls` (1 .. 2^20) replaces the kernels' limit, which is
 * about a second.  `ws` is a prepared workspace with room for at least one
 * tile; `res` (device) receives GPUTF_TIMEOUT, position 0, written 0, and the
 * workspace is left ready for the next call, as after any call that timed
 * out.  Enqueued on `stream`; faults nothing, allocates nothing. */
gputf_status gputf_test_wait_timeout(void *ws, size_t ws_bytes, int which, uint32_t polls, gputf_result *res,
                                     cudaStream_t stream);

/* Names of codes, for messages. */
const char *gputf_error_name(int32_t error);
const char *gputf_status_name(gputf_status status);
/* The last CUDA error code seen by a call on this thread (0 if none). */
int gputf_last_cuda_error(void);
/* Library version: major * 10000 + minor * 100 + patch. */
int gputf_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GPUTF_H */
