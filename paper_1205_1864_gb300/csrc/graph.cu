// CUDA graph construction: conditional WHILE nodes inside stream capture and
// the per-handle cache of instantiated solve graphs.
#include "graph.cuh"

namespace sghsc {

static int eager_while(sg_problem* h, cudaStream_t s, const EnqueueCond& pre, const EnqueueCond& body) {
  if (h->loop_depth >= 8) {
    set_error("eager loop: nested too deeply");
    return SG_ERR_UNSUPPORTED;
  }
  LoopCtl lc{0, 0, h->loopflags + h->loop_depth};
  ++h->loop_depth;
  int r = pre(s, lc);
  while (r == SG_OK) {
    cudaError_t e = cudaMemcpyAsync(h->loopflag_host, lc.flag, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      set_error("eager loop: %s", cudaGetErrorString(e));
      r = SG_ERR_CUDA;
      break;
    }
    if (!*h->loopflag_host) break;
    r = body(s, lc);
  }
  --h->loop_depth;
  return r;
}

int capture_while(sg_problem* h, cudaStream_t s, const EnqueueCond& pre, const EnqueueCond& body) {
  if (!h->capturing) return eager_while(h, s, pre, body);
  if (h->cap_depth + 1 >= (int)(sizeof(h->cap) / sizeof(h->cap[0]))) {
    set_error("graph capture: loops nested too deeply");
    return SG_ERR_UNSUPPORTED;
  }
  cudaStreamCaptureStatus st;
  cudaGraph_t g = nullptr;
  SG_TRY_CUDA(cudaStreamGetCaptureInfo(s, &st, nullptr, &g, nullptr, nullptr, nullptr));
  if (st != cudaStreamCaptureStatusActive || !g) {
    set_error("graph capture: stream is not capturing");
    return SG_ERR_CUDA;
  }
  cudaGraphConditionalHandle cond;
  SG_TRY_CUDA(cudaGraphConditionalHandleCreate(&cond, g, 0, 0));
  const LoopCtl lc{cond, 1, nullptr};
  SG_TRY(pre(s, lc));
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  SG_TRY_CUDA(cudaStreamGetCaptureInfo(s, &st, nullptr, &g, &deps, nullptr, &ndeps));
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = cond;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  SG_TRY_CUDA(cudaGraphAddNode(&node, g, deps, nullptr, ndeps, &np));
  cudaGraph_t bodyg = np.conditional.phGraph_out[0];
  cudaStream_t bs = h->cap[++h->cap_depth];
  SG_TRY_CUDA(cudaStreamBeginCaptureToGraph(bs, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  int r = body(bs, lc);
  cudaGraph_t out = nullptr;
  cudaError_t e = cudaStreamEndCapture(bs, &out);
  --h->cap_depth;
  if (r != SG_OK) return r;
  SG_TRY_CUDA(e);
  SG_TRY_CUDA(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  return SG_OK;
}

void clear_graphs(sg_problem* h) {
  ++h->ws_gen;
  for (auto& kv : h->graphs) {
    cudaGraphExecDestroy(kv.second.exec);
    cudaGraphDestroy(kv.second.graph);
  }
  h->graphs.clear();
}

int run_graph(sg_problem* h, const std::string& key, const Enqueue& build, cudaStream_t launch) {
  if (h->eager) {
    h->loop_depth = 0;
    return build(launch);
  }
  auto it = h->graphs.find(key);
  if (it == h->graphs.end()) {
    cudaStream_t cs = h->cap[0];
    h->cap_depth = 0;
    h->capturing = true;
    SG_TRY_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
    int r = build(cs);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(cs, &g);
    h->capturing = false;
    if (r != SG_OK) {
      if (g) cudaGraphDestroy(g);
      return r;
    }
    SG_TRY_CUDA(e);
    cudaGraphExec_t ex;
    cudaError_t ei = cudaGraphInstantiate(&ex, g, 0);
    if (ei != cudaSuccess) {
      cudaGraphDestroy(g);
      SG_TRY_CUDA(ei);
    }
    it = h->graphs.emplace(key, GraphEntry{g, ex}).first;
  }
  SG_TRY_CUDA(cudaGraphLaunch(it->second.exec, launch));
  return SG_OK;
}

}  // namespace sghsc
