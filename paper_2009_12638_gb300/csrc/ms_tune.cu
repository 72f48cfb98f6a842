// ms_tune.cu -- launch-shape heuristics (see ms_tune.h).
#include <algorithm>

#include "ms_tune.h"

namespace ms {

static int max_clusters(Tuner& t, int prec, int mode, int threads, int cluster, int* out) {
  auto key = std::make_tuple(prec, mode, threads, cluster);
  auto it = t.occ.find(key);
  if (it != t.occ.end()) {
    *out = it->second;
    return 0;
  }
  cudaError_t e = mode == 1 ? async_max_clusters(prec, threads, cluster, out)
                            : sweep_max_clusters(prec, threads, cluster, out);
  if (e != cudaSuccess) return (int)e;
  t.occ[key] = *out;
  return 0;
}

int choose_shape(Tuner& t, int prec, int mode, const std::vector<Task>& tasks, long long maxpts, int req_cluster,
                 int req_threads, int req_slots, LaunchShape* out) {
  const int ntasks = (int)tasks.size();
  double mean_bz = 0.0, mean_plane = 0.0;
  for (const Task& k : tasks) {
    mean_bz += k.bz;
    mean_plane += (double)k.bx * k.by;
  }
  mean_bz /= std::max(1, ntasks);
  mean_plane /= std::max(1, ntasks);
  LaunchShape s;
  s.threads = req_threads ? req_threads : (mean_plane >= 2048 ? 512 : 256);
  if (req_cluster) {
    s.cluster = req_cluster;
  } else {
    int c = (int)(mean_bz / 6.0);
    s.cluster = std::max(1, std::min(8, c));
  }
  int maxc = 0;
  int e = max_clusters(t, prec, mode, s.threads, s.cluster, &maxc);
  if (e) return e;
  if (maxc < 1) return (int)cudaErrorInvalidConfiguration;
  if (req_slots) {
    s.slots = std::min(req_slots, maxc);
  } else {
    int g = std::min(maxc, ntasks);
    if (prec == 1) {
      // keep the CG vectors of the blocks in flight inside L2 (~80 MB usable)
      const double per = 4.0 * (double)maxpts * 4.0;
      int l2cap = (int)std::max(1.0, 80.0e6 / per);
      int fill = (152 + s.cluster - 1) / s.cluster;
      g = std::min(g, std::max(l2cap, fill));
    }
    s.slots = std::max(1, g);
  }
  *out = s;
  return 0;
}

}  // namespace ms
