// ms_tune.h -- launch-shape selection for the sweep kernels: CTAs per block
// (cluster size), threads per CTA and blocks in flight (cluster slots).
#pragma once
#include <cuda_runtime.h>

#include <map>
#include <tuple>
#include <vector>

#include "ms_internal.h"

namespace ms {

struct LaunchShape {
  int cluster = 1;
  int threads = 512;
  int slots = 1;
  int variant = -1;   // >= 0: resident engine variant (ms_resident.cu); -1: streaming engine;
                      // -2: vectorised FP32 streaming engine (ms_stream4.cu)
  size_t smem = 0;    // dynamic shared memory bytes (resident engine)
  double est = 0.0;   // model estimate used to rank shapes before measuring
};

struct Tuner {
  // cache of maxActiveClusters per (kernel kind, smem, threads, cluster)
  std::map<std::tuple<int, int, int, int>, int> occ;
  // measured best shape per problem signature (see signature())
  std::map<std::vector<long long>, LaunchShape> best;
  // sync mode, resident engine: measured ms per sweep of the persistent
  // dataflow launch and of the per-sweep graph, per signature + shape (< 0: not yet)
  struct ModeMs {
    double flow = -1.0, sweep = -1.0;
  };
  std::map<std::vector<long long>, ModeMs> mode_ms;
  void release() {
    occ.clear();
    best.clear();
    mode_ms.clear();
  }
};

// Problem signature for the cache of measured shapes: precision, mode,
// engine request, and the sorted multiset of block shapes.
std::vector<long long> signature(int prec, int mode, int engine, const std::vector<Task>& tasks);

// Every launchable shape for the problem, best model estimate first (the
// resident engine's shapes, when it applies, precede the streaming ones).
// Explicit non-zero requests restrict the list.  Returns a cudaError_t value.
// req_variant >= 0 keeps only that row of the resident variant table.
int list_shapes(Tuner& t, int prec, int mode, int engine, const std::vector<Task>& tasks, long long maxpts,
                int req_cluster, int req_threads, int req_slots, int req_variant, std::vector<LaunchShape>* out);

// The first shape of list_shapes.
int choose_shape(Tuner& t, int prec, int mode, int engine, const std::vector<Task>& tasks, long long maxpts,
                 int req_cluster, int req_threads, int req_slots, int req_variant, LaunchShape* out);

}  // namespace ms
