// graph.cu -- CUDA-graph capture of fused (or unfused) launch sequences.
//
// A caller brackets any sequence of hf_launch / hf_launch_single calls on a
// stream (plus other streams joined to it with events) by hf_graph_begin and
// hf_graph_end; the recorded work replays with one hf_graph_launch.  This is
// how an N-way persistent fused kernel -- or the serial and multi-stream
// baselines it is compared with -- become a single submission.
#include "kernels.cuh"

namespace hf {
hf_status set_last_error(hf_status s, const char *msg);   // runtime.cu
}

struct hf_graph_t {
    cudaGraph_t graph;
    cudaGraphExec_t exec;
};

extern "C" {

hf_status hf_graph_begin(void *stream)
{
    cudaError_t e = cudaStreamBeginCapture(static_cast<cudaStream_t>(stream), cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return hf::set_last_error(HF_ERR_CUDA, cudaGetErrorString(e));
    return HF_OK;
}

hf_status hf_graph_end(void *stream, hf_graph *out)
{
    if (!out) return hf::set_last_error(HF_ERR_INVALID, "NULL output");
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(static_cast<cudaStream_t>(stream), &g);
    if (e != cudaSuccess) return hf::set_last_error(HF_ERR_CUDA, cudaGetErrorString(e));
    cudaGraphExec_t x = nullptr;
    e = cudaGraphInstantiate(&x, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return hf::set_last_error(HF_ERR_CUDA, cudaGetErrorString(e));
    }
    *out = new hf_graph_t{g, x};
    return HF_OK;
}

hf_status hf_graph_launch(hf_graph g, void *stream)
{
    if (!g) return hf::set_last_error(HF_ERR_INVALID, "NULL graph");
    cudaError_t e = cudaGraphLaunch(g->exec, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return hf::set_last_error(HF_ERR_CUDA, cudaGetErrorString(e));
    return HF_OK;
}

void hf_graph_destroy(hf_graph g)
{
    if (!g) return;
    cudaGraphExecDestroy(g->exec);
    cudaGraphDestroy(g->graph);
    delete g;
}

} // extern "C"
