// Reusable CUDA graphs of a batch of library calls, and sequence lengths from offsets.
//
// A batch's launches (count -> rank -> partition on a plan from host-side bounds)
// contain no host synchronisation, so they can be recorded by stream capture. Each
// capture gets a topology signature: its nodes in order (type, and for kernel
// nodes the function) and its edges (ends and type, programmatic or full). A capture whose signature matches one
// of the handle's instantiated graphs updates that graph in place
// (cudaGraphExecUpdate: same kernels, new parameters: other buffers, sizes and
// grids); any other capture is instantiated. The signature check matters: a
// single-set batch and a multi-set batch launch different preparation kernels in
// the same number of nodes, and an in-place update between them is accepted by
// the runtime but does not run the new kernels' dependencies correctly.
#include <cuda_runtime.h>

#include <new>
#include <vector>

#include "sad_common.cuh"

using namespace sad;

namespace {

struct GraphEntry {
  std::vector<uintptr_t> sig;  // per node: type (and kernel function); per edge: ends, type
  size_t edges = 0;
  cudaGraphExec_t exec = nullptr;
  int kernels = 0;
  uint64_t last_use = 0;
};

constexpr size_t kMaxExecs = 4;

}  // namespace

struct sad_graph_s {
  std::vector<GraphEntry> entries;
  int current = -1;            // entry the next launch runs
  uint64_t clock = 0;
  int64_t updates = 0;         // captures applied by update
  int64_t instantiations = 0;  // captures that needed a new instantiation
};

namespace {

int graph_check(cudaError_t e) { return e == cudaSuccess ? SAD_OK : SAD_ERR_CUDA; }

bool graph_aligned(const void *p, size_t a) { return reinterpret_cast<uintptr_t>(p) % a == 0; }

__global__ void lengths_kernel(const int64_t *__restrict__ offsets, int32_t n,
                               int32_t *__restrict__ lengths, WsHeader *hdr) {
  pdl_enter();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t l = offsets[i + 1] - offsets[i];
    if (l < 0 || l > 0x7FFFFFFF) {
      if (hdr) record_error(hdr, SAD_ERR_BAD_INPUT, (int)i);
      lengths[i] = 0;
    } else {
      lengths[i] = (int32_t)l;
    }
  }
}

}  // namespace

extern "C" {

int sad_seq_lengths(const int64_t *d_offsets, int32_t n_seq, int32_t *d_lengths, void *d_ws,
                    void *stream) {
  if (n_seq < 0 || (n_seq > 0 && (!d_offsets || !d_lengths))) return SAD_ERR_INVALID_ARGUMENT;
  if (d_ws && !graph_aligned(d_ws, 256)) return SAD_ERR_INVALID_ARGUMENT;
  if (n_seq == 0) return SAD_OK;
  const int64_t blocks = (n_seq + 255) / 256;
  pdl_launch(lengths_kernel, (unsigned)(blocks < 4096 ? blocks : 4096), 256, 0,
             static_cast<cudaStream_t>(stream), d_offsets, n_seq, d_lengths,
             static_cast<WsHeader *>(d_ws));
  SAD_LAUNCH_CHECK();
  return SAD_OK;
}

int sad_graph_begin(void *stream) {
  return graph_check(
      cudaStreamBeginCapture(static_cast<cudaStream_t>(stream), cudaStreamCaptureModeThreadLocal));
}

int sad_graph_end(void *stream, sad_graph *g) {
  cudaGraph_t graph = nullptr;
  int rc = graph_check(cudaStreamEndCapture(static_cast<cudaStream_t>(stream), &graph));
  if (rc) return rc;
  if (!g) {
    cudaGraphDestroy(graph);
    return SAD_ERR_INVALID_ARGUMENT;
  }
  if (!*g) {
    *g = new (std::nothrow) sad_graph_s();
    if (!*g) {
      cudaGraphDestroy(graph);
      return SAD_ERR_CUDA;
    }
  }
  sad_graph_s &G = **g;
  // the capture's signature
  GraphEntry e;
  size_t n_nodes = 0;
  rc = graph_check(cudaGraphGetNodes(graph, nullptr, &n_nodes));
  std::vector<cudaGraphNode_t> nodes(n_nodes);
  if (!rc && n_nodes) rc = graph_check(cudaGraphGetNodes(graph, nodes.data(), &n_nodes));
  for (size_t i = 0; !rc && i < n_nodes; ++i) {
    cudaGraphNodeType t;
    rc = graph_check(cudaGraphNodeGetType(nodes[i], &t));
    if (rc) break;
    e.sig.push_back((uintptr_t)t);
    if (t == cudaGraphNodeTypeKernel) {
      cudaKernelNodeParams kp;
      rc = graph_check(cudaGraphKernelNodeGetParams(nodes[i], &kp));
      e.sig.push_back(reinterpret_cast<uintptr_t>(kp.func));
      ++e.kernels;
    }
  }
  // edges: (from, to, type) by node position
  if (!rc) rc = graph_check(cudaGraphGetEdges(graph, nullptr, nullptr, nullptr, &e.edges));
  if (!rc && e.edges) {
    std::vector<cudaGraphNode_t> from(e.edges), to(e.edges);
    std::vector<cudaGraphEdgeData> data(e.edges);
    size_t ne = e.edges;
    rc = graph_check(cudaGraphGetEdges(graph, from.data(), to.data(), data.data(), &ne));
    auto pos = [&](cudaGraphNode_t v) {
      for (size_t i = 0; i < n_nodes; ++i)
        if (nodes[i] == v) return (uintptr_t)i;
      return ~(uintptr_t)0;
    };
    for (size_t i = 0; !rc && i < ne; ++i) {
      e.sig.push_back(pos(from[i]));
      e.sig.push_back(pos(to[i]));
      e.sig.push_back((uintptr_t)data[i].type | ((uintptr_t)data[i].from_port << 8) |
                      ((uintptr_t)data[i].to_port << 16));
    }
  }
  if (rc) {
    cudaGraphDestroy(graph);
    return rc;
  }
  G.clock += 1;
  for (size_t k = 0; k < G.entries.size(); ++k) {
    GraphEntry &x = G.entries[k];
    if (x.sig != e.sig || x.edges != e.edges) continue;
    cudaGraphExecUpdateResultInfo info;
    if (cudaGraphExecUpdate(x.exec, graph, &info) == cudaSuccess) {
      cudaGraphDestroy(graph);
      x.last_use = G.clock;
      G.current = (int)k;
      G.updates += 1;
      return SAD_OK;
    }
    // refused after all: this entry is replaced by the new instantiation
    (void)cudaGetLastError();
    cudaGraphExecDestroy(x.exec);
    G.entries.erase(G.entries.begin() + (long)k);
    break;
  }
  rc = graph_check(cudaGraphInstantiate(&e.exec, graph, 0));
  cudaGraphDestroy(graph);
  if (rc) return rc;
  if (G.entries.size() >= kMaxExecs) {
    // drop the least recently used instantiation
    size_t lru = 0;
    for (size_t k = 1; k < G.entries.size(); ++k)
      if (G.entries[k].last_use < G.entries[lru].last_use) lru = k;
    cudaGraphExecDestroy(G.entries[lru].exec);
    G.entries.erase(G.entries.begin() + (long)lru);
  }
  e.last_use = G.clock;
  G.entries.push_back(std::move(e));
  G.current = (int)G.entries.size() - 1;
  G.instantiations += 1;
  return SAD_OK;
}

int sad_graph_launch(sad_graph g, void *stream) {
  if (!g || g->current < 0) return SAD_ERR_INVALID_ARGUMENT;
  const GraphEntry &e = g->entries[(size_t)g->current];
  const int rc = graph_check(cudaGraphLaunch(e.exec, static_cast<cudaStream_t>(stream)));
  if (rc == SAD_OK) note_launch(e.kernels);
  return rc;
}

int sad_graph_stats(sad_graph g, int64_t *updates, int64_t *instantiations, int32_t *kernels) {
  if (!g || !updates || !instantiations || !kernels) return SAD_ERR_INVALID_ARGUMENT;
  *updates = g->updates;
  *instantiations = g->instantiations;
  *kernels = g->current >= 0 ? g->entries[(size_t)g->current].kernels : 0;
  return SAD_OK;
}

int sad_graph_destroy(sad_graph g) {
  if (!g) return SAD_OK;
  for (GraphEntry &e : g->entries)
    if (e.exec) cudaGraphExecDestroy(e.exec);
  delete g;
  return SAD_OK;
}

}  // extern "C"
