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

static long long res_smem_bytes(const std::vector<Task>& tasks, int zs) {
  long long ps = 0;
  for (const Task& k : tasks) ps = std::max(ps, (long long)(k.by + 2) * (4 * ((k.bx + 3) / 4) + 8));
  return (zs + 4) * ps * 4;
}

// Resident engine: every block must fit the variant at cluster size c.
static bool res_fits(const std::vector<Task>& tasks, int nt, int kc, int zs, int c) {
  for (const Task& k : tasks) {
    if (k.bz < c) return false;
    if ((k.bz + c - 1) / c > zs) return false;
    if ((long long)((k.bx + 3) / 4) * k.by > (long long)kc * nt) return false;
  }
  return true;
}

static int choose_resident(Tuner& t, const std::vector<Task>& tasks, long long maxpts, int req_cluster,
                           int req_threads, int req_slots, LaunchShape* out) {
  const int ntasks = (int)tasks.size();
  double best = 1e300;
  bool found = false;
  for (int v = 0; v < res_variant_count(); ++v) {
    int nt, kc, zs;
    res_variant_info(v, &nt, &kc, &zs);
    if (req_threads && req_threads != nt) continue;
    const long long smem = res_smem_bytes(tasks, zs);
    if (smem > 200 * 1024) continue;
    for (int c = 1; c <= kMaxCluster; ++c) {
      if (req_cluster && c != req_cluster) continue;
      if (!res_fits(tasks, nt, kc, zs, c)) continue;
      auto key = std::make_tuple(100 + v, (int)smem, nt, c);
      int occ = 0;
      auto it = t.occ.find(key);
      if (it != t.occ.end()) {
        occ = it->second;
      } else {
        if (res_max_clusters(v, c, (size_t)smem, &occ) != cudaSuccess) {
          cudaGetLastError();
          occ = 0;
        }
        t.occ[key] = occ;
      }
      if (occ < 1) continue;
      const int slots = req_slots ? std::min(req_slots, occ) : std::min(occ, ntasks);
      // rounds of the task queue x points each CTA handles per round
      const double rounds = std::ceil((double)ntasks / slots);
      const double est = rounds * ((double)maxpts / c) * (1.0 + 0.02 * c);
      if (est < best) {
        best = est;
        found = true;
        out->variant = v;
        out->cluster = c;
        out->threads = nt;
        out->slots = slots;
        out->smem = (size_t)smem;
      }
    }
  }
  return found ? 0 : -1;
}

int choose_shape(Tuner& t, int prec, int mode, int engine, const std::vector<Task>& tasks, long long maxpts,
                 int req_cluster, int req_threads, int req_slots, LaunchShape* out) {
  const int ntasks = (int)tasks.size();
  if (prec == 1 && mode == 0 && engine != 1) {
    LaunchShape r;
    if (choose_resident(t, tasks, maxpts, req_cluster, req_threads, req_slots, &r) == 0) {
      *out = r;
      return 0;
    }
    if (engine == 2) return (int)cudaErrorInvalidConfiguration;  // resident requested but nothing fits
  }
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
