// Loop driver: device-controlled iteration without host round-trips (Sec. 2.1: every
// host<->device transfer costs a PCI-Express latency; on GB300 the analogue is the kernel
// launch latency, hidden here by replaying the iteration as a CUDA graph whose WHILE node
// is cleared by the kernel that detects convergence).
#include <cstring>

#include "pk_internal.cuh"

namespace pk {

static pk_status add_while(cudaGraph_t graph, cudaGraphConditionalHandle h, const cudaGraphNode_t* deps,
                           size_t ndeps, cudaGraphNode_t* node, cudaGraph_t* body);

__global__ void k_enable_cond(DevState* st, cudaGraphConditionalHandle h) {
  st->use_cond = 1;
  st->cond = h;
}

static pk_status build_graph(pk_csr* A, const LoopSpec& L, pk_graph_entry* g) {
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  g->exec = nullptr;
  g->graph = nullptr;
  g->kind = -1;
  cudaGraph_t graph;
  PK_CUDA(cudaGraphCreate(&graph, 0));
  cudaGraphConditionalHandle h;
  PK_CUDA(cudaGraphConditionalHandleCreate(&h, graph, 1u, cudaGraphCondAssignDefault));
  cudaGraphNode_t node;
  cudaGraph_t body;
  pk_status pe = add_while(graph, h, nullptr, 0, &node, &body);
  if (pe) { cudaGraphDestroy(graph); return pe; }
  PK_CUDA(cudaStreamBeginCaptureToGraph(A->cap_stream, body, nullptr, nullptr, 0,
                                        cudaStreamCaptureModeThreadLocal));
  for (int u = 0; u < L.unroll; ++u) L.body(A->cap_stream, nullptr);
  cudaGraph_t captured;
  cudaError_t ce = cudaStreamEndCapture(A->cap_stream, &captured);
  if (ce != cudaSuccess) {
    cudaGraphDestroy(graph);
    return cuda_fail(ce, "cudaStreamEndCapture");
  }
  cudaGraphExec_t exec;
  ce = cudaGraphInstantiate(&exec, graph, 0);
  if (ce != cudaSuccess) {
    cudaGraphDestroy(graph);
    return cuda_fail(ce, "cudaGraphInstantiate");
  }
  g->graph = graph;
  g->exec = exec;
  g->kind = L.kind;
  for (int k = 0; k < 4; ++k) {
    g->key[k] = L.keys[k];
    g->ikey[k] = L.ikeys[k];
  }
  g->body_kernels = L.body_kernels;
  g->cond_handle = h;
  return PK_OK;
}

__global__ void k_enable_cond2(DevState* st, cudaGraphConditionalHandle h,
                               cudaGraphConditionalHandle h2) {
  st->use_cond = 1;
  st->cond = h;
  st->cond2 = h2;
}

void launch_enable_cond2(pk_csr* A, const pk_graph_entry* g, cudaStream_t s) {
  k_enable_cond2<<<1, 1, 0, s>>>(A->st, g->cond_handle, g->cond2_handle);
}

static pk_status add_while(cudaGraph_t graph, cudaGraphConditionalHandle h, const cudaGraphNode_t* deps,
                           size_t ndeps, cudaGraphNode_t* node, cudaGraph_t* body) {
  // cudaGraphNodeParams has no usable default constructor in C++: zero raw storage instead
  alignas(cudaGraphNodeParams) unsigned char raw[sizeof(cudaGraphNodeParams)];
  memset(raw, 0, sizeof(raw));
  cudaGraphNodeParams* cp = reinterpret_cast<cudaGraphNodeParams*>(raw);
  cp->type = cudaGraphNodeTypeConditional;
  cp->conditional.handle = h;
  cp->conditional.type = cudaGraphCondTypeWhile;
  cp->conditional.size = 1;
  PK_CUDA(cudaGraphAddNode(node, graph, deps, nullptr, ndeps, cp));
  *body = cp->conditional.phGraph_out[0];
  return PK_OK;
}

pk_status build_nested_graph(pk_csr* A, int kind, const void* const keys[4], const int64_t ikeys[4],
                             const std::function<void(cudaStream_t)>& pre,
                             const std::function<void(cudaStream_t)>& body,
                             const std::function<void(cudaStream_t)>& post, pk_graph_entry** out) {
  for (auto& e : A->graphs) {
    if (e.kind == kind && e.key[0] == keys[0] && e.key[1] == keys[1] && e.key[2] == keys[2] &&
        e.key[3] == keys[3] && e.ikey[0] == ikeys[0] && e.ikey[1] == ikeys[1] &&
        e.ikey[2] == ikeys[2] && e.ikey[3] == ikeys[3]) {
      *out = &e;
      return PK_OK;
    }
  }
  pk_graph_entry* g = nullptr;
  for (auto& e : A->graphs) if (e.kind == kind) { g = &e; break; }
  if (!g) for (auto& e : A->graphs) if (e.kind < 0) { g = &e; break; }
  if (!g) g = &A->graphs[0];
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  g->exec = nullptr;
  g->graph = nullptr;
  g->kind = -1;
  pk_status e;
  cudaGraph_t graph;
  PK_CUDA(cudaGraphCreate(&graph, 0));
  cudaGraphConditionalHandle ho, hi;
  PK_CUDA(cudaGraphConditionalHandleCreate(&ho, graph, 1u, cudaGraphCondAssignDefault));
  cudaGraphNode_t wo;
  cudaGraph_t bo;
  if ((e = add_while(graph, ho, nullptr, 0, &wo, &bo))) { cudaGraphDestroy(graph); return e; }
  // the inner condition is set explicitly by the kernels every cycle
  PK_CUDA(cudaGraphConditionalHandleCreate(&hi, bo, 0u, 0));
  // pre() into the outer body, remembering its tail nodes
  PK_CUDA(cudaStreamBeginCaptureToGraph(A->cap_stream, bo, nullptr, nullptr, 0,
                                        cudaStreamCaptureModeThreadLocal));
  pre(A->cap_stream);
  cudaStreamCaptureStatus cs;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  PK_CUDA(cudaStreamGetCaptureInfo(A->cap_stream, &cs, nullptr, nullptr, &deps, nullptr, &ndeps));
  cudaGraphNode_t tail[8];
  if (ndeps > 8) { set_error("nested graph: too many tail nodes"); return PK_ERR_CUDA; }
  for (size_t k = 0; k < ndeps; ++k) tail[k] = deps[k];
  cudaGraph_t tmp;
  PK_CUDA(cudaStreamEndCapture(A->cap_stream, &tmp));
  cudaGraphNode_t wi;
  cudaGraph_t bi;
  if ((e = add_while(bo, hi, tail, ndeps, &wi, &bi))) { cudaGraphDestroy(graph); return e; }
  PK_CUDA(cudaStreamBeginCaptureToGraph(A->cap_stream, bi, nullptr, nullptr, 0,
                                        cudaStreamCaptureModeThreadLocal));
  body(A->cap_stream);
  PK_CUDA(cudaStreamEndCapture(A->cap_stream, &tmp));
  PK_CUDA(cudaStreamBeginCaptureToGraph(A->cap_stream, bo, &wi, nullptr, 1,
                                        cudaStreamCaptureModeThreadLocal));
  post(A->cap_stream);
  PK_CUDA(cudaStreamEndCapture(A->cap_stream, &tmp));
  cudaGraphExec_t exec;
  cudaError_t ce = cudaGraphInstantiate(&exec, graph, 0);
  if (ce != cudaSuccess) {
    cudaGraphDestroy(graph);
    return cuda_fail(ce, "cudaGraphInstantiate(nested)");
  }
  g->graph = graph;
  g->exec = exec;
  g->kind = kind;
  for (int k = 0; k < 4; ++k) {
    g->key[k] = keys[k];
    g->ikey[k] = ikeys[k];
  }
  g->cond_handle = ho;
  g->cond2_handle = hi;
  *out = g;
  return PK_OK;
}

pk_status run_loop(pk_csr* A, const pk_opts* o, cudaStream_t s, const LoopSpec& L, Timer* T,
                   int* launches) {
  const bool timing = T && T->on;
  if (o->loop != PK_LOOP_HOST && !timing) {
    pk_graph_entry* g = nullptr;
    for (auto& e : A->graphs) {
      if (e.kind == L.kind && e.key[0] == L.keys[0] && e.key[1] == L.keys[1] &&
          e.key[2] == L.keys[2] && e.key[3] == L.keys[3] && e.ikey[0] == L.ikeys[0] &&
          e.ikey[1] == L.ikeys[1] && e.ikey[2] == L.ikeys[2] && e.ikey[3] == L.ikeys[3]) {
        g = &e;
        break;
      }
    }
    if (!g) {
      // reuse the slot of the same kind, else the first free / oldest slot
      for (auto& e : A->graphs) if (e.kind == L.kind) { g = &e; break; }
      if (!g) for (auto& e : A->graphs) if (e.kind < 0) { g = &e; break; }
      if (!g) g = &A->graphs[0];
      pk_status st = build_graph(A, L, g);
      if (st) return st;
    }
    k_enable_cond<<<1, 1, 0, s>>>(A->st, g->cond_handle);
    PK_CUDA(cudaGetLastError());
    PK_CUDA(cudaGraphLaunch(g->exec, s));
    *launches += 1;  // k_enable_cond; body kernels are added from the pass count
    return PK_OK;
  }
  // host-driven loop
  const int every = timing ? 1 : (o->check_every > 0 ? o->check_every : 16);
  for (;;) {
    for (int k = 0; k < every; ++k) {
      L.body(s, timing ? T : nullptr);
      *launches += L.body_kernels;
    }
    PK_CUDA(cudaGetLastError());
    if (timing) {
      pk_status e = T->flush();
      if (e) return e;
    }
    int done = 0;
    PK_CUDA(cudaMemcpyAsync(&A->st_host->done, &A->st->done, sizeof(int), cudaMemcpyDeviceToHost, s));
    PK_CUDA(cudaStreamSynchronize(s));
    done = A->st_host->done;
    if (done) break;
  }
  return PK_OK;
}

}  // namespace pk
