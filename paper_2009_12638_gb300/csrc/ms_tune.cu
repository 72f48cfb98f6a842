// ms_tune.cu -- launch-shape heuristics (see ms_tune.h).
#include <algorithm>

#include "ms_resident_variants.h"
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

static long long res_smem_bytes(const std::vector<Task>& tasks, int zs, int ds) {
  long long mx = 0;
  for (const Task& k : tasks) mx = std::max(mx, res_smem_floats(k.bx, k.by, zs, ds != 0));
  return mx * 4;
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

static void list_resident(Tuner& t, int mode, const std::vector<Task>& tasks, long long maxpts, int req_cluster,
                          int req_threads, int req_slots, int req_variant, std::vector<LaunchShape>* out) {
  const int ntasks = (int)tasks.size();
  for (int v = 0; v < res_variant_count(); ++v) {
    if (req_variant >= 0 && v != req_variant) continue;
    int nt, kc, zs, ds, qr;
    res_variant_info(v, &nt, &kc, &zs, &ds, &qr);
    if (req_threads && req_threads != nt) continue;
    const long long smem = res_smem_bytes(tasks, zs, ds);
    if (smem > 220 * 1024) continue;
    for (int c = 1; c <= kMaxCluster; ++c) {
      if (req_cluster && c != req_cluster) continue;
      if (!res_fits(tasks, nt, kc, zs, c)) continue;
      auto key = std::make_tuple(100 + v + 1000 * mode, (int)smem, nt, c);
      int occ = 0;
      auto it = t.occ.find(key);
      if (it != t.occ.end()) {
        occ = it->second;
      } else {
        if (res_max_clusters(v, c, (size_t)smem, &occ, mode == 1) != cudaSuccess) {
          cudaGetLastError();
          occ = 0;
        }
        t.occ[key] = occ;
      }
      if (occ < 1) continue;
      LaunchShape r;
      r.variant = v;
      r.cluster = c;
      r.threads = nt;
      r.slots = req_slots ? std::min(req_slots, occ) : std::min(occ, ntasks);
      r.smem = (size_t)smem;
      // rounds of the task queue x points each CTA handles per round
      const double rounds = std::ceil((double)ntasks / r.slots);
      // QR: one stencil per iteration.  The asynchronous kernel (never timed by
      // the tuner) holds more state: with q in registers it spills at 512 and
      // 1024 threads (measured 5% slower at 256^3), so there QR only pays at
      // <= 256 threads (measured 27% faster at 128^3)
      // The single-reduction CG (qr 2) halves the cluster sums per iteration but
      // moves d to shared memory and reads more of it per iteration: measured
      // 4.02 vs 3.01 ms per 256^3 sweep against the best q-in-registers row, so
      // it ranks behind the two-reduction rows and is kept where it measures faster.
      const double qr_factor =
          qr == 2 ? 1.1 : (!qr ? 1.0 : (mode == 1 && nt > 256 ? 1.05 : 0.85));
      r.est = rounds * ((double)maxpts / c) * (1.0 + 0.02 * c) * qr_factor;
      out->push_back(r);
    }
  }
}

static int streaming_shape(Tuner& t, int prec, int mode, const std::vector<Task>& tasks, long long maxpts,
                           int req_cluster, int req_threads, int req_slots, int threads, LaunchShape* out) {
  const int ntasks = (int)tasks.size();
  double mean_bz = 0.0;
  for (const Task& k : tasks) mean_bz += k.bz;
  mean_bz /= std::max(1, ntasks);
  LaunchShape s;
  s.threads = req_threads ? req_threads : threads;
  s.cluster = req_cluster ? req_cluster : std::max(1, std::min(8, (int)(mean_bz / 6.0)));
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
      const int l2cap = (int)std::max(1.0, 80.0e6 / per);
      const int fill = (152 + s.cluster - 1) / s.cluster;
      g = std::min(g, std::max(l2cap, fill));
    }
    s.slots = std::max(1, g);
  }
  s.variant = -1;
  s.est = 4.0 * std::ceil((double)ntasks / s.slots) * ((double)maxpts / s.cluster);  // ~4x slower than on chip
  *out = s;
  return 0;
}

std::vector<long long> signature(int prec, int mode, int engine, const std::vector<Task>& tasks) {
  std::vector<long long> sig = {prec, mode, engine, (long long)tasks.size()};
  std::vector<long long> shapes;
  for (const Task& k : tasks) shapes.push_back(((long long)k.bx << 40) | ((long long)k.by << 20) | k.bz);
  std::sort(shapes.begin(), shapes.end());
  sig.insert(sig.end(), shapes.begin(), shapes.end());
  return sig;
}

int list_shapes(Tuner& t, int prec, int mode, int engine, const std::vector<Task>& tasks, long long maxpts,
                int req_cluster, int req_threads, int req_slots, int req_variant, std::vector<LaunchShape>* out) {
  out->clear();
  if (prec == 1 && engine != 1) {
    list_resident(t, mode, tasks, maxpts, req_cluster, req_threads, req_slots, req_variant, out);
    std::stable_sort(out->begin(), out->end(),
                     [](const LaunchShape& a, const LaunchShape& b) { return a.est < b.est; });
    if (engine == 2) return out->empty() ? (int)cudaErrorInvalidConfiguration : 0;
  }
  int last = 0;
  if (mode == 0) {
    // vectorised streaming candidates (sync; FP32 inner solve or FP64): same slot model as the scalar engine
    for (int threads : {512, 1024}) {
      if (req_threads && req_threads != threads) continue;
      LaunchShape s;
      if (streaming_shape(t, prec, mode, tasks, maxpts, req_cluster, 0, req_slots, threads, &s) != 0) continue;
      int occ = 0;
      auto key = std::make_tuple(300 + prec, 0, threads, s.cluster);
      auto it = t.occ.find(key);
      if (it != t.occ.end()) {
        occ = it->second;
      } else {
        if (strip_max_clusters(prec, threads, s.cluster, &occ) != cudaSuccess) {
          cudaGetLastError();
          occ = 0;
        }
        t.occ[key] = occ;
      }
      if (occ < 1) continue;
      s.threads = threads;
      s.slots = std::min(s.slots, occ);
      s.variant = -2;
      s.est *= 0.6;  // fewer, wider loads than the scalar streaming engine
      out->push_back(s);
    }
  }
  for (int threads : {512, 1024}) {
    if (req_threads && req_threads != threads && threads != 512) continue;
    LaunchShape s;
    last = streaming_shape(t, prec, mode, tasks, maxpts, req_cluster, req_threads, req_slots, threads, &s);
    if (last == 0) out->push_back(s);
    if (req_threads) break;
  }
  return out->empty() ? (last ? last : (int)cudaErrorInvalidConfiguration) : 0;
}

int choose_shape(Tuner& t, int prec, int mode, int engine, const std::vector<Task>& tasks, long long maxpts,
                 int req_cluster, int req_threads, int req_slots, int req_variant, LaunchShape* out) {
  std::vector<LaunchShape> all;
  const int rc = list_shapes(t, prec, mode, engine, tasks, maxpts, req_cluster, req_threads, req_slots, req_variant,
                             &all);
  if (rc) return rc;
  *out = all.front();
  return 0;
}

}  // namespace ms
