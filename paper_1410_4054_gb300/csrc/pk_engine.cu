// Loop driver: device-controlled iteration without host round-trips (Sec. 2.1: every
// host<->device transfer costs a PCI-Express latency; on GB300 the analogue is the kernel
// launch latency, hidden here by replaying the iteration as a CUDA graph whose WHILE node
// is cleared by the kernel that detects convergence).
#include <cstring>

#include "pk_internal.cuh"

namespace pk {

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
  // cudaGraphNodeParams has no usable default constructor in C++: zero raw storage instead
  alignas(cudaGraphNodeParams) unsigned char raw[sizeof(cudaGraphNodeParams)];
  memset(raw, 0, sizeof(raw));
  cudaGraphNodeParams* cp = reinterpret_cast<cudaGraphNodeParams*>(raw);
  cp->type = cudaGraphNodeTypeConditional;
  cp->conditional.handle = h;
  cp->conditional.type = cudaGraphCondTypeWhile;
  cp->conditional.size = 1;
  cudaGraphNode_t node;
  PK_CUDA(cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, cp));
  cudaGraph_t body = cp->conditional.phGraph_out[0];
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

pk_status run_loop(pk_csr* A, const pk_opts* o, cudaStream_t s, const LoopSpec& L, Timer* T,
                   int* launches) {
  const bool timing = T && T->on;
  if (o->loop == PK_LOOP_GRAPH && !timing) {
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
