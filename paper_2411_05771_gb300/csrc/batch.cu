// Batched persistent schedule: one operator (A_S, A_S^T, B_S, B_S^T, H or
// the FBP A_S^dagger = (pi/m) B_S H of Sec. 2.1) applied to many instances
// at once - images of different sizes, each with its own angle list and its
// own sketch S (Eq. (e:skeiloss): every sample and transform of a step may
// draw a different S_k, Algorithm 2).
//
// The host cuts every instance into the tasks of the operator's kernel (a
// block of angles of an image group for A and B^T, an 8 x 128 tile of an
// image group for A^T and B, a sinogram row for H; groups of 4 images share
// their positions and weights), sorts them by decreasing cost, and uploads
// the list once.  A run is one persistent launch per kernel: as many CTAs (or
// 8-CTA clusters) as fit on the GPU at once take tasks from a global counter
// until none is left, so large and small instances share the machine without
// a tail of idle SMs.  Every output element is still produced by exactly one
// task, in the same order as the single-instance launches, so the results are
// deterministic and bitwise equal to calling the operator per instance.
//
// skei_batch_tune times the candidate task shapes (angles per band task) and
// worker counts on the caller's stream and keeps the fastest.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"

using namespace skei;

namespace {

constexpr int kFilterKernel = 100;  // phase kernel id of the Ram-Lak rows
constexpr int kBandMaxAB = 8;

struct Phase {
  int kernel = 0;                  // OP_* or kFilterKernel
  std::vector<BatchItem> items;    // host copies, pointers already final
  BatchItem *d_items = nullptr;
  int4 *d_tasks = nullptr;
  int *d_queue = nullptr;          // [2]
  int n_tasks = 0, cap_tasks = 0;
  int block = 0;                   // band: angles per task; tile/filter: CTAs per SM
  int workers = 0;                 // CTAs (tile, filter) or clusters (band)
  size_t smem = 0;
};

}  // namespace

struct skei_batch_s {
  int op = -1, device = -1;
  std::vector<Phase> phases;
  float *d_work = nullptr;         // FBP: filtered sinograms (FP32)
  bool tuned = false;
};

namespace {

int sm_count_dev() {
  int dev = 0, c = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev);
  return c > 0 ? c : 1;
}

bool is_band(int k) { return k == OP_JOSEPH || k == OP_BP_ADJ; }
bool is_tile(int k) { return k == OP_JOSEPH_ADJ || k == OP_BACKPROJECT; }

// Task list of a phase for `block` (band: angles per task), sorted by
// decreasing cost; ties keep item / image / position order.
void make_tasks(const Phase &ph, int block, std::vector<int4> *tasks) {
  struct T {
    double cost;
    int4 t;
  };
  std::vector<T> v;
  int tr = 0, tc = 0;
  tile_batch_shape(&tr, &tc);
  for (int q = 0; q < (int)ph.items.size(); ++q) {
    const BatchItem &it = ph.items[q];
    if (is_band(ph.kernel)) {
      for (int gi = 0; gi < n_groups(it.B); ++gi) {
        int b0, ni;
        group_at(it.B, gi, &b0, &ni);
        for (int a0 = 0; a0 < it.m; a0 += block) {
          const int na = std::min(block, it.m - a0);
          v.push_back({(double)ni * na * it.n_det * it.N, make_int4(q, b0 << 3 | ni, a0, 0)});
        }
      }
    } else if (is_tile(ph.kernel)) {
      for (int gi = 0; gi < n_groups(it.B); ++gi) {
        int b0, ni;
        group_at(it.B, gi, &b0, &ni);
        for (int ty = 0; ty * tr < it.N; ++ty)
          for (int tx = 0; tx * tc < it.N; ++tx) {
            const int rows = std::min(tr, it.N - ty * tr), cols = std::min(tc, it.N - tx * tc);
            v.push_back({(double)ni * it.m * rows * cols, make_int4(q, b0 << 3 | ni, ty, tx)});
          }
      }
    } else {
      for (int r = 0; r < it.B * it.m; ++r)
        v.push_back({(double)it.n_det * it.n_det, make_int4(q, r, 0, 0)});
    }
  }
  std::stable_sort(v.begin(), v.end(), [](const T &a, const T &b) { return a.cost > b.cost; });
  tasks->resize(v.size());
  for (size_t i = 0; i < v.size(); ++i) (*tasks)[i] = v[i].t;
}

// Shared memory and worker count of a phase for `block`.
int phase_shape(const Phase &ph, int block, size_t *smem, int *workers, int *max_per_sm) {
  if (is_band(ph.kernel)) {
    size_t s = 0;
    for (const BatchItem &it : ph.items) {
      if (it.B >= 4)
        s = std::max(s, band_batch_smem(ph.kernel, it.N, it.n_det, it.n_angles, block, 4));
      if (it.B & 3)
        s = std::max(s, band_batch_smem(ph.kernel, it.N, it.n_det, it.n_angles, block, 1));
    }
    if (s > 227 * 1024)
      return set_error(SKEI_EINVAL, "batch: %d angles per task need %zu bytes of shared memory",
                       block, s);
    int clusters = 0;
    SKEI_TRY(band_batch_occupancy(ph.kernel, s, &clusters));
    *smem = s;
    *workers = clusters;
    if (max_per_sm) *max_per_sm = 0;
    return SKEI_OK;
  }
  int per_sm = 0;
  if (is_tile(ph.kernel)) {
    SKEI_TRY(tile_batch_occupancy(ph.kernel, &per_sm));
    *smem = 0;
  } else {
    int nd = 1;
    for (const BatchItem &it : ph.items) nd = std::max(nd, it.n_det);
    *smem = filter_batch_smem(nd);
    SKEI_TRY(filter_batch_occupancy(*smem, &per_sm));
  }
  if (max_per_sm) *max_per_sm = per_sm;
  const int k = block > 0 ? std::min(block, per_sm) : per_sm;
  *workers = sm_count_dev() * k;
  return SKEI_OK;
}

// Builds and uploads the task list of `block` (synchronous: never inside a
// stream capture).
int configure(Phase &ph, int block) {
  std::vector<int4> tasks;
  make_tasks(ph, block, &tasks);
  if (tasks.size() > (size_t)0x7fffffff) return set_error(SKEI_EINVAL, "batch: too many tasks");
  size_t smem = 0;
  int workers = 0;
  SKEI_TRY(phase_shape(ph, block, &smem, &workers, nullptr));
  if ((int)tasks.size() > ph.cap_tasks) {
    if (ph.d_tasks) cudaFree(ph.d_tasks);
    ph.d_tasks = nullptr;
    ph.cap_tasks = 0;
    cudaError_t e = dev_malloc(reinterpret_cast<void **>(&ph.d_tasks), tasks.size() * sizeof(int4));
    if (e != cudaSuccess) return set_error(SKEI_ENOMEM, "batch: task list of %zu tasks", tasks.size());
    ph.cap_tasks = (int)tasks.size();
  }
  cudaError_t e = cudaMemcpy(ph.d_tasks, tasks.data(), tasks.size() * sizeof(int4),
                             cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_error(e, "batch: task upload");
  ph.n_tasks = (int)tasks.size();
  ph.block = block;
  ph.workers = std::max(1, std::min(workers, ph.n_tasks));
  ph.smem = smem;
  return SKEI_OK;
}

int run_phase(const Phase &ph, cudaStream_t st) {
  if (is_band(ph.kernel))
    return launch_band_batch_op(ph.kernel, ph.d_items, ph.d_tasks, ph.n_tasks, ph.block, ph.smem,
                                ph.workers, ph.d_queue, st);
  if (is_tile(ph.kernel))
    return launch_tile_batch_op(ph.kernel, ph.d_items, ph.d_tasks, ph.n_tasks, ph.workers,
                                ph.d_queue, st);
  return launch_filter_batch(ph.d_items, ph.d_tasks, ph.n_tasks, ph.smem, ph.workers,
                             ph.d_queue, st);
}

// Greedy list-scheduling estimate of a band phase's time with `ab` angles
// per task on `clusters` workers: tasks in decreasing cost order, each to the
// worker that frees first.  A task costs its ray-line samples plus the
// staging of its image band (about twice a sample per staged pixel).
double band_makespan(const Phase &ph, int ab, int clusters) {
  std::vector<double> cost;
  for (const BatchItem &it : ph.items)
    for (int gi = 0; gi < n_groups(it.B); ++gi) {
      int b0, ni;
      group_at(it.B, gi, &b0, &ni);
      for (int a0 = 0; a0 < it.m; a0 += ab) {
        const int na = std::min(ab, it.m - a0);
        cost.push_back(ni * ((double)na * it.n_det * it.N + 2.0 * it.N * it.N));
      }
    }
  std::sort(cost.begin(), cost.end(), [](double a, double b) { return a > b; });
  std::vector<double> load((size_t)std::max(clusters, 1), 0.0);
  for (double c : cost) {
    auto w = std::min_element(load.begin(), load.end());
    *w += c;
  }
  return *std::max_element(load.begin(), load.end());
}

// Default angles per band task: the smallest estimated time (ties to the
// larger block: less staging).  Tile and filter phases: 0 (all resident
// CTAs).
int default_block(const Phase &ph) {
  if (!is_band(ph.kernel)) return 0;
  int best = 1;
  double best_t = 1e300;
  int m_max = 1;
  for (const BatchItem &it : ph.items) m_max = std::max(m_max, it.m);
  for (int ab = 1; ab <= std::min(kBandMaxAB, m_max); ++ab) {
    size_t smem = 0;
    int clusters = 0;
    if (phase_shape(ph, ab, &smem, &clusters, nullptr) != SKEI_OK) continue;
    const double t = band_makespan(ph, ab, clusters);
    if (t <= best_t) { best_t = t; best = ab; }
  }
  return best;
}

void free_batch(skei_batch b) {
  for (Phase &ph : b->phases) {
    if (ph.d_items) cudaFree(ph.d_items);
    if (ph.d_tasks) cudaFree(ph.d_tasks);
    if (ph.d_queue) cudaFree(ph.d_queue);
  }
  if (b->d_work) cudaFree(b->d_work);
  delete b;
}

int make_phase(skei_batch b, int kernel, std::vector<BatchItem> items) {
  Phase ph;
  ph.kernel = kernel;
  ph.items = std::move(items);
  b->phases.push_back(ph);
  Phase &p = b->phases.back();
  cudaError_t e = dev_malloc(reinterpret_cast<void **>(&p.d_items), p.items.size() * sizeof(BatchItem));
  if (e != cudaSuccess) return set_error(SKEI_ENOMEM, "batch: item table");
  e = cudaMemcpy(p.d_items, p.items.data(), p.items.size() * sizeof(BatchItem),
                 cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_error(e, "batch: item upload");
  e = dev_malloc(reinterpret_cast<void **>(&p.d_queue), 2 * sizeof(int));
  if (e != cudaSuccess) return set_error(SKEI_ENOMEM, "batch: work queue");
  e = cudaMemset(p.d_queue, 0, 2 * sizeof(int));
  if (e != cudaSuccess) return cuda_error(e, "batch: work queue reset");
  return configure(p, default_block(p));
}

}  // namespace

extern "C" {

int skei_batch_create(int op, const skei_batch_item *items, int n_items, skei_batch *out) {
  SKEI_RANGE("skei_batch_create");
  if (!out) return set_error(SKEI_EINVAL, "out is NULL");
  *out = nullptr;
  if (op < SKEI_BATCH_PROJ_FWD || op > SKEI_BATCH_FBP)
    return set_error(SKEI_EINVAL, "unknown batch operator %d", op);
  if (!items || n_items < 1 || n_items > SKEI_MAX_BATCH_ITEMS)
    return set_error(SKEI_EINVAL, "n_items=%d outside [1, %d]", n_items, SKEI_MAX_BATCH_ITEMS);
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return set_error(SKEI_ECUDA, "no current device");
  size_t work_floats = 0;
  for (int q = 0; q < n_items; ++q) {
    const skei_batch_item &s = items[q];
    SKEI_TRY(check_plan(s.plan));
    if (s.plan->device != dev)
      return set_error(SKEI_EINVAL, "item %d: its plan lives on device %d, current is %d", q,
                       s.plan->device, dev);
    SKEI_TRY(check_dtype(s.dtype_in));
    SKEI_TRY(check_dtype(s.dtype_out));
    SKEI_TRY(check_batch(s.B));
    SKEI_TRY(check_dev_ptr(s.in, "item.in"));
    SKEI_TRY(check_dev_ptr(s.out, "item.out"));
    SKEI_TRY(check_idx(s.plan, s.idx, s.m));
    if (op == SKEI_BATCH_FBP) work_floats += (size_t)s.B * s.m * s.plan->n_det;
  }

  skei_batch b = new skei_batch_s;
  b->op = op;
  b->device = dev;
  if (op == SKEI_BATCH_FBP) {
    cudaError_t e = dev_malloc(reinterpret_cast<void **>(&b->d_work),
                               std::max<size_t>(work_floats, 4) * sizeof(float));
    if (e != cudaSuccess) {
      free_batch(b);
      return set_error(SKEI_ENOMEM, "batch: FBP workspace of %zu floats", work_floats);
    }
  }
  auto item = [&](const skei_batch_item &s, const void *in, int in_bf16, void *o, int out_bf16,
                  float alpha) {
    return BatchItem{s.plan->d_ang, s.plan->d_status, in, o, s.idx, s.plan->N, s.plan->n_det,
                     s.plan->n_angles, s.m, s.B, alpha, in_bf16, out_bf16};
  };
  std::vector<BatchItem> first, second;
  size_t off = 0;
  for (int q = 0; q < n_items; ++q) {
    const skei_batch_item &s = items[q];
    const int ib = s.dtype_in == SKEI_BF16, ob = s.dtype_out == SKEI_BF16;
    if (op == SKEI_BATCH_FBP) {
      float *w = b->d_work + off;
      off += (size_t)s.B * s.m * s.plan->n_det;
      first.push_back(item(s, s.in, ib, w, 0, (float)(s.scale * M_PI / s.m)));
      second.push_back(item(s, w, 0, s.out, ob, 1.0f));
    } else {
      first.push_back(item(s, s.in, ib, s.out, ob, s.scale));
    }
  }
  static const int kernel_of[] = {OP_JOSEPH, OP_JOSEPH_ADJ, OP_BACKPROJECT, OP_BP_ADJ,
                                  kFilterKernel, kFilterKernel};
  int rc = make_phase(b, kernel_of[op], std::move(first));
  if (!rc && op == SKEI_BATCH_FBP) rc = make_phase(b, OP_BACKPROJECT, std::move(second));
  if (rc) {
    free_batch(b);
    return rc;
  }
  *out = b;
  return SKEI_OK;
}

int skei_batch_run(skei_batch b, void *stream) {
  SKEI_RANGE("skei_batch_run");
  if (!b) return set_error(SKEI_EINVAL, "batch is NULL");
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != b->device)
    return set_error(SKEI_EINVAL, "batch was created on device %d, current is %d", b->device, dev);
  for (const Phase &ph : b->phases) SKEI_TRY(run_phase(ph, reinterpret_cast<cudaStream_t>(stream)));
  return SKEI_OK;
}

namespace {

// On-disk tuning cache (file named by SKEI_AUTOTUNE_CACHE): one line per tuned
// phase, "<signature>\t<block>", the signature naming the device, the phase's
// kernel and every item's shape and storage types.  A phase whose signature
// is in the file takes the recorded block without timing; newly tuned phases
// are appended (one short write each).
std::string phase_signature(const Phase &ph) {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp prop{};
  cudaGetDeviceProperties(&prop, dev);
  std::string sig = std::string(prop.name) + "/sm" + std::to_string(prop.multiProcessorCount) +
                    "/k" + std::to_string(ph.kernel) + ":";
  for (const BatchItem &it : ph.items) {
    char buf[96];
    std::snprintf(buf, sizeof buf, "%dx%dx%dx%dx%d%s%s,", it.N, it.n_det, it.n_angles, it.m,
                  it.B, it.in_bf16 ? "h" : "f", it.out_bf16 ? "h" : "f");
    sig += buf;
  }
  for (char &c : sig)
    if (c == '\t' || c == '\n') c = ' ';
  return sig;
}

// The block recorded for `sig` in the cache file (the last matching line),
// or 0.
int cache_lookup(const char *path, const std::string &sig) {
  FILE *f = std::fopen(path, "r");
  if (!f) return 0;
  int found = 0;
  std::string line;
  int ch;
  while (true) {
    line.clear();
    while ((ch = std::fgetc(f)) != EOF && ch != '\n') line.push_back((char)ch);
    const size_t tab = line.rfind('\t');
    if (tab != std::string::npos && line.compare(0, tab, sig) == 0 && tab == sig.size()) {
      const int v = std::atoi(line.c_str() + tab + 1);
      if (v > 0) found = v;
    }
    if (ch == EOF) break;
  }
  std::fclose(f);
  return found;
}

void cache_store(const char *path, const std::string &sig, int block) {
  FILE *f = std::fopen(path, "a");
  if (!f) return;   // a cache that cannot be written only costs the next tuning
  const std::string line = sig + "\t" + std::to_string(block) + "\n";
  std::fwrite(line.data(), 1, line.size(), f);
  std::fclose(f);
}

}  // namespace

int skei_batch_tune(skei_batch b, int reps, void *stream) {
  SKEI_RANGE("skei_batch_tune");
  if (!b) return set_error(SKEI_EINVAL, "batch is NULL");
  if (reps < 1 || reps > 1000) return set_error(SKEI_EINVAL, "reps=%d outside [1, 1000]", reps);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) == cudaSuccess && cap != cudaStreamCaptureStatusNone)
    return set_error(SKEI_EINVAL, "skei_batch_tune synchronises: call it outside a capture");
  // earlier runs of this batch may still read the task lists on `stream`
  cudaError_t se = cudaStreamSynchronize(st);
  if (se != cudaSuccess) return cuda_error(se, "tune: stream synchronise");
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return set_error(SKEI_ECUDA, "tune: event");
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return set_error(SKEI_ECUDA, "tune: event");
  }
  int rc = SKEI_OK;
  const char *cache = std::getenv("SKEI_AUTOTUNE_CACHE");
  if (cache && !*cache) cache = nullptr;
  for (Phase &ph : b->phases) {
    std::string sig;
    if (cache) {
      sig = phase_signature(ph);
      const int cached = cache_lookup(cache, sig);
      if (cached > 0 && configure(ph, cached) == SKEI_OK) continue;
    }
    std::vector<int> cands;
    if (is_band(ph.kernel)) {
      int m_max = 1;
      for (const BatchItem &it : ph.items) m_max = std::max(m_max, it.m);
      for (int ab : {1, 2, 3, 4, 6, 8})
        if (ab <= std::min(kBandMaxAB, m_max)) cands.push_back(ab);
    } else {
      size_t smem = 0;
      int workers = 0, max_k = 1;
      if ((rc = phase_shape(ph, 0, &smem, &workers, &max_k))) break;
      for (int k = 1; k <= max_k; k *= 2) cands.push_back(k);
      if (cands.back() != max_k) cands.push_back(max_k);
    }
    float best_ms = 1e30f;
    int best = ph.block;
    for (int c : cands) {
      if (configure(ph, c) != SKEI_OK) continue;  // e.g. too much shared memory
      if ((rc = run_phase(ph, st))) break;        // warm-up
      cudaEventRecord(e0, st);
      for (int r = 0; r < reps && !rc; ++r) rc = run_phase(ph, st);
      cudaEventRecord(e1, st);
      if (rc) break;
      cudaError_t e = cudaEventSynchronize(e1);
      if (e != cudaSuccess) { rc = cuda_error(e, "tune: timing"); break; }
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best_ms) { best_ms = ms; best = c; }
    }
    if (rc) break;
    if ((rc = configure(ph, best))) break;
    if (cache) cache_store(cache, sig, best);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!rc) b->tuned = true;
  return rc;
}

int skei_batch_info(skei_batch b, int phase, int *n_phases, int *n_tasks, int *workers,
                    int *block) {
  if (!b) return set_error(SKEI_EINVAL, "batch is NULL");
  if (n_phases) *n_phases = (int)b->phases.size();
  if (phase < 0 || phase >= (int)b->phases.size())
    return set_error(SKEI_EINVAL, "phase %d outside [0, %zu)", phase, b->phases.size());
  const Phase &ph = b->phases[phase];
  if (n_tasks) *n_tasks = ph.n_tasks;
  if (workers) *workers = ph.workers;
  if (block) *block = ph.block;
  return SKEI_OK;
}

int skei_batch_destroy(skei_batch b) {
  SKEI_RANGE("skei_batch_destroy");
  if (!b) return SKEI_OK;
  free_batch(b);
  return SKEI_OK;
}

}  // extern "C"
