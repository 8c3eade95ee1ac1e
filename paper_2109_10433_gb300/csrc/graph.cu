/*
 * CUDA-graph capture of batched launches: a batch's launch is recorded once
 * and replayed, so a serving loop or a repeated batch pays one graph launch
 * instead of the host-side argument checks and kernel launch each time.
 */
#include <new>

#include <cuda_runtime.h>

#include "gputf.h"

struct gputf_graph {
    cudaGraph_t graph;
    cudaGraphExec_t exec;
};

extern "C" gputf_status gputf_batch_graph_create(const gputf_batch *utf8_to_utf16,
                                                 const gputf_batch *utf16_to_utf8, int config, void *ws,
                                                 size_t ws_bytes, cudaStream_t stream, gputf_graph **graph)
{
    if (graph == nullptr || stream == nullptr) return GPUTF_STATUS_INVALID_ARGUMENT;
    *graph = nullptr;
    cudaStreamCaptureStatus capturing = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(stream, &capturing) != cudaSuccess || capturing != cudaStreamCaptureStatusNone)
        return GPUTF_STATUS_INVALID_ARGUMENT;
    /* checks (and the one-time device query) outside the capture */
    if (gputf_batch_workspace_bytes(utf8_to_utf16 ? utf8_to_utf16->units : 0,
                                    utf8_to_utf16 ? utf8_to_utf16->count : 0,
                                    utf16_to_utf8 ? utf16_to_utf8->units : 0,
                                    utf16_to_utf8 ? utf16_to_utf8->count : 0) > ws_bytes)
        return GPUTF_STATUS_WORKSPACE_TOO_SMALL;
    if (cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return GPUTF_STATUS_CUDA_ERROR;
    const gputf_status st = gputf_batch_transcode(utf8_to_utf16, utf16_to_utf8, config, ws, ws_bytes, stream);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(stream, &g);
    if (st != GPUTF_STATUS_OK || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return st != GPUTF_STATUS_OK ? st : GPUTF_STATUS_CUDA_ERROR;
    }
    cudaGraphExec_t exec = nullptr;
    if (cudaGraphInstantiate(&exec, g, 0) != cudaSuccess) {
        cudaGraphDestroy(g);
        return GPUTF_STATUS_CUDA_ERROR;
    }
    gputf_graph *h = new (std::nothrow) gputf_graph{g, exec};
    if (h == nullptr) {
        cudaGraphExecDestroy(exec);
        cudaGraphDestroy(g);
        return GPUTF_STATUS_CUDA_ERROR;
    }
    *graph = h;
    return GPUTF_STATUS_OK;
}

extern "C" gputf_status gputf_graph_launch(gputf_graph *graph, cudaStream_t stream)
{
    if (graph == nullptr) return GPUTF_STATUS_INVALID_ARGUMENT;
    return cudaGraphLaunch(graph->exec, stream) == cudaSuccess ? GPUTF_STATUS_OK : GPUTF_STATUS_CUDA_ERROR;
}

extern "C" void gputf_graph_destroy(gputf_graph *graph)
{
    if (graph == nullptr) return;
    cudaGraphExecDestroy(graph->exec);
    cudaGraphDestroy(graph->graph);
    delete graph;
}
