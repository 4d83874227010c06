// CUDA-graph replay of fixed launch sequences (a V-cycle, one solver
// iteration).  A sequence is identified by a key that fixes every launch in
// it (the level, precision, cycle shape and the vector pointers); its first
// use runs directly (kernel attributes and occupancy are settled on the way),
// its second is captured on the mesh's private stream (the legacy stream
// cannot capture) and every use from then on is one graph launch on the
// caller's stream.  Anything that changes the launches of a level (a sweep
// split, the FP64 arithmetic mode, the coefficient) clears the cache.  While
// launch profiling is on, or while the caller's stream is being captured
// into a graph of its own, sequences run directly.
#include <map>

#include "hhg_internal.h"

namespace hhg {

struct GraphCache {
  struct Entry {
    int uses = 0;
    cudaGraphExec_t exec = nullptr;
  };
  std::map<GraphKey, Entry> entries;
  cudaStream_t capture = nullptr;
};

namespace {
constexpr size_t kMaxGraphs = 64;   // cached sequences per mesh; the cache is cleared beyond this

void drop_all(GraphCache& gc) {
  for (auto& e : gc.entries)
    if (e.second.exec) cudaGraphExecDestroy(e.second.exec);
  gc.entries.clear();
}
}  // namespace

void graphs_create(Mesh& m) {
  m.graphs = new GraphCache();
  check_cuda(cudaStreamCreateWithFlags(&m.graphs->capture, cudaStreamNonBlocking), "capture stream");
}

void graphs_destroy(Mesh& m) {
  if (!m.graphs) return;
  drop_all(*m.graphs);
  if (m.graphs->capture) cudaStreamDestroy(m.graphs->capture);
  delete m.graphs;
  m.graphs = nullptr;
}

void graphs_clear(const Mesh& m) {
  if (m.graphs) drop_all(*m.graphs);
}

void graphed(const Mesh& m, const GraphKey& key, cudaStream_t st, const std::function<void(cudaStream_t)>& body) {
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  const cudaError_t ce = cudaStreamIsCapturing(st, &cap);
  if (ce != cudaSuccess) cudaGetLastError();
  if (!m.graphs || profiling_on() || ce != cudaSuccess || cap != cudaStreamCaptureStatusNone) {
    body(st);   // the caller's stream is itself being captured: its own graph takes the launches
    return;
  }
  GraphCache& gc = *m.graphs;
  auto it = gc.entries.find(key);
  if (it == gc.entries.end()) {
    if (gc.entries.size() >= kMaxGraphs) drop_all(gc);
    it = gc.entries.emplace(key, GraphCache::Entry{}).first;
  }
  GraphCache::Entry& e = it->second;
  if (!e.exec && e.uses++ == 0) {
    body(st);
    return;
  }
  if (!e.exec) {
    cudaGraph_t graph = nullptr;
    check_cuda(cudaStreamBeginCapture(gc.capture, cudaStreamCaptureModeThreadLocal), "begin capture");
    try {
      body(gc.capture);
    } catch (...) {
      cudaStreamEndCapture(gc.capture, &graph);
      if (graph) cudaGraphDestroy(graph);
      gc.entries.erase(it);
      throw;
    }
    check_cuda(cudaStreamEndCapture(gc.capture, &graph), "end capture");
    const cudaError_t ie = cudaGraphInstantiate(&e.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) {
      gc.entries.erase(it);
      check_cuda(ie, "graph instantiate");
    }
  }
  check_cuda(cudaGraphLaunch(e.exec, st), "graph launch");
}

}  // namespace hhg
