// C ABI of CUDA-graph capture and joining (many instances in one launch).
#include "context.h"

using namespace sccsd;

// ======================================================================
// CUDA graphs of the right transformation (many instances in one launch)
// ======================================================================
extern "C" {

int sccsd_capture_transform(sccsd_ctx* c, int side, int nvec, const double* R, double* sigma,
                            void** graph) {
  if (!c) return SCCSD_EINVAL;
  if (!R || !sigma || !graph || nvec < 1 || (side != 0 && side != 1))
    return fail(c, SCCSD_EINVAL, "bad capture arguments");
  if (!c->cur) return fail(c, SCCSD_ESTATE, "call sccsd_residual first");
  if (!c->be->is_device(R) || !c->be->is_device(sigma))
    return fail(c, SCCSD_EINVAL, "capture needs device vectors");
  if (c->be->stream() == nullptr)
    return fail(c, SCCSD_EINVAL, "capture needs a context created with a (non-default) stream");
  cudaStream_t st = (cudaStream_t)c->be->stream();
  return guarded(c, [&] {
    // warm-up with the same targets: sizes every buffer and pool slot the
    // captured launches use, converts the state-dependent operands once
    transform(c, side, nvec, R, sigma);
    c->be->sync();
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      throw CudaError("cudaStreamBeginCapture failed");
    cudaGraph_t g = nullptr;
    try {
      c->be->set_capturing(true);
      transform(c, side, nvec, R, sigma);
      c->be->set_capturing(false);
    } catch (...) {
      c->be->set_capturing(false);
      cudaStreamEndCapture(st, &g);
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      throw;
    }
    if (cudaStreamEndCapture(st, &g) != cudaSuccess || !g) throw CudaError("cudaStreamEndCapture failed");
    *graph = (void*)g;
  });
}

int sccsd_graph_join(void** graphs, int n, void** exec) {
  if (!graphs || n < 1 || !exec) return SCCSD_EINVAL;
  cudaGraph_t parent = nullptr;
  if (cudaGraphCreate(&parent, 0) != cudaSuccess) return SCCSD_ECUDA;
  for (int k = 0; k < n; ++k) {
    cudaGraphNode_t node;
    if (!graphs[k] ||
        cudaGraphAddChildGraphNode(&node, parent, nullptr, 0, (cudaGraph_t)graphs[k]) != cudaSuccess) {
      cudaGraphDestroy(parent);
      cudaGetLastError();
      return SCCSD_ECUDA;
    }
  }
  cudaGraphExec_t e = nullptr;
  cudaError_t r = cudaGraphInstantiate(&e, parent, 0);
  cudaGraphDestroy(parent);
  if (r != cudaSuccess) {
    cudaGetLastError();
    return SCCSD_ECUDA;
  }
  *exec = (void*)e;
  return SCCSD_OK;
}

int sccsd_graph_launch(void* exec, void* stream) {
  if (!exec) return SCCSD_EINVAL;
  if (cudaGraphLaunch((cudaGraphExec_t)exec, (cudaStream_t)stream) != cudaSuccess) {
    cudaGetLastError();
    return SCCSD_ECUDA;
  }
  return SCCSD_OK;
}

void sccsd_graph_destroy(void* graph) {
  if (graph) cudaGraphDestroy((cudaGraph_t)graph);
}

void sccsd_graph_exec_destroy(void* exec) {
  if (exec) cudaGraphExecDestroy((cudaGraphExec_t)exec);
}

}  // extern "C"
