// tqr_tune.cu -- the measured tile-size autotuner (tqr_autotune_run and the
// table behind tqr_autotune).
//
// The paper's tile size b and inner block (Sections 3.1-3.2) trade the
// efficiency of the update kernels against the length of the panel chain;
// for a batch of many small and medium matrices the best pair depends on the
// matrix size.  Matrices are grouped into size classes by ceil(log2 m) and
// ceil(log2 n); for a class the tuner factors a batch of copies of one
// representative matrix (the geometric middle of the class) with every
// candidate (nb, ib), times each batch on the device, and keeps the fastest
// per matrix.  tqr_autotune then answers from this table and falls back to
// the fixed rule for classes never tuned.  The table can be saved to and
// loaded from a text file, one class per line.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "tqr.h"
#include "tqr_api_internal.h"

namespace tqr {

struct TuneEntry {
  int nb, ib;
  double us_per_matrix;
};

static std::mutex g_tmu;
static std::map<std::pair<int, int>, TuneEntry> g_table;

static int ceil_log2(int64_t x) {
  int b = 0;
  while ((int64_t(1) << b) < x) ++b;
  return b;
}

std::pair<int, int> tune_class(int64_t m, int64_t n) { return {ceil_log2(std::max<int64_t>(1, m)),
                                                                 ceil_log2(std::max<int64_t>(1, n))}; }

bool tune_lookup(int64_t m, int64_t n, int* nb, int* ib) {
  std::lock_guard<std::mutex> lk(g_tmu);
  auto it = g_table.find(tune_class(m, n));
  if (it == g_table.end()) return false;
  *nb = it->second.nb;
  *ib = it->second.ib;
  return true;
}

// Candidate (nb, ib) pairs for a class whose matrices are at most mx on
// their longer side: nb from {16, 32, 64, 96, 128, 192, 256} up to the
// smallest that holds mx, ib in {8, 16, 32} dividing nb.
static std::vector<std::pair<int, int>> candidates(int64_t mx) {
  std::vector<std::pair<int, int>> out;
  for (int nb : {16, 32, 64, 96, 128, 192, 256}) {
    for (int ib : {8, 16, 32}) {
      if (ib > nb || nb % ib != 0) continue;
      int cs, occ, smem;
      if (!choose_shape(nb, ib, 8, &cs, &occ, &smem)) continue;
      out.push_back({nb, ib});
    }
    if (nb >= mx) break;
  }
  return out;
}

// Deterministic fill: a counter hash mapped to [-1, 1) (the tuner needs a
// full-rank matrix of the class's size, not a particular distribution).
__global__ void tune_fill(double* A, long long count) {
  for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < count;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    unsigned long long z = static_cast<unsigned long long>(e) * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    A[e] = static_cast<double>(z >> 11) * 0x1p-52 - 1.0;
  }
}

}  // namespace tqr

using namespace tqr;

extern "C" int tqr_autotune_run(int64_t m, int64_t n, void* stream) {
  if (m < 1 || m > (1 << 20)) return -1;
  if (n < 1 || n > (1 << 20)) return -2;
  const std::pair<int, int> cls = tune_class(m, n);
  {
    std::lock_guard<std::mutex> lk(g_tmu);
    if (g_table.count(cls)) return TQR_OK;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // representative matrix: the geometric middle of the class's ranges
  auto mid = [](int b) {
    const double lo = b > 0 ? std::ldexp(1.0, b - 1) + 1 : 1.0, hi = std::ldexp(1.0, b);
    return static_cast<int64_t>(std::llround(std::sqrt(lo * hi)));
  };
  const int64_t mr = mid(cls.first), nr = mid(cls.second);
  const double flops = mr >= nr ? 2.0 * mr * nr * nr - 2.0 * nr * nr * nr / 3.0
                                : 2.0 * nr * mr * mr - 2.0 * mr * mr * mr / 3.0;
  // enough copies for ~1e11 flops (8 .. 1024): a batch in the throughput
  // regime, as inside a large mixed batch -- a few copies of a large matrix
  // would measure its critical path instead and favour small tiles
  const int count = static_cast<int>(std::max(8.0, std::min(1024.0, std::ceil(1e11 / std::max(flops, 1.0)))));
  const size_t elems = static_cast<size_t>(mr) * nr;
  size_t tmax = 0;
  const auto cands = candidates(std::max(mr, nr));
  for (const auto& c : cands) tmax = std::max(tmax, tqr_t_size(mr, nr, c.first, c.second));
  double *A = nullptr, *T = nullptr;
  if (lib_malloc(reinterpret_cast<void**>(&A), sizeof(double) * elems * count, st) != cudaSuccess ||
      lib_malloc(reinterpret_cast<void**>(&T), tmax * count, st) != cudaSuccess) {
    cudaGetLastError();
    if (A) cudaFreeAsync(A, st);
    return TQR_ERR_NOMEM;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  std::vector<tqr_desc> d(count);
  TuneEntry best = {0, 0, INFINITY};
  int status = TQR_OK;
  for (const auto& c : cands) {
    const size_t tsz = tqr_t_size(mr, nr, c.first, c.second) / sizeof(double);
    for (int a = 0; a < count; ++a) {
      d[a].m = mr;
      d[a].n = nr;
      d[a].A = A + elems * a;
      d[a].lda = mr;
      d[a].T = T + tsz * a;
      d[a].nb = c.first;
      d[a].ib = c.second;
    }
    float ms_best = INFINITY;
    for (int rep = 0; rep < 2 && status == TQR_OK; ++rep) {  // the first builds the plan and graph
      tune_fill<<<1024, 256, 0, st>>>(A, static_cast<long long>(elems) * count);
      uint64_t ticket = 0;
      cudaEventRecord(e0, st);
      int s = tqr_batch_submit(count, d.data(), &ticket, st);
      if (s == TQR_OK) s = tqr_batch_wait(ticket, nullptr);
      cudaEventRecord(e1, st);
      if (s != TQR_OK || cudaEventSynchronize(e1) != cudaSuccess) {
        status = s != TQR_OK ? s : TQR_ERR_CUDA;
        break;
      }
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0) ms_best = std::min(ms_best, ms);
    }
    if (status != TQR_OK) break;
    const double us = 1e3 * ms_best / count;
    if (us < best.us_per_matrix) best = {c.first, c.second, us};
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(A, st);
  cudaFreeAsync(T, st);
  cudaStreamSynchronize(st);
  if (status != TQR_OK) return status;
  std::lock_guard<std::mutex> lk(g_tmu);
  g_table[cls] = best;
  return TQR_OK;
}

// ---------------------------------------------------------------- batch-level tuning
// Candidate tile policies for a whole batch, each a map from a matrix's size
// class to (nb, ib): the fixed rule, the rule with ib 8, the per-class table
// of tqr_autotune_run, that table with ib 16, and the table for matrices of
// at most 512 rows and columns with the rule above.  The batch's own shapes
// are factored under each, and the fastest policy's choices are written into
// the class table.
static void rule_tiles(int64_t m, int64_t n, int* nb, int* ib) {
  const int64_t mx = std::max(m, n);
  int b = 16;
  while (b < 128 && b < mx) b *= 2;
  *nb = b;
  *ib = std::min(16, b);
}

extern "C" int tqr_autotune_batch(int count, const int64_t* ms, const int64_t* ns, void* stream) {
  if (count < 1) return -1;
  if (ms == nullptr) return -2;
  if (ns == nullptr) return -3;
  for (int a = 0; a < count; ++a)
    if (ms[a] < 1 || ns[a] < 1 || ms[a] > (1 << 20) || ns[a] > (1 << 20)) return -2;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // the per-class measurements first (each class once)
  std::map<std::pair<int, int>, std::pair<int64_t, int64_t>> classes;
  for (int a = 0; a < count; ++a) classes.emplace(tune_class(ms[a], ns[a]), std::make_pair(ms[a], ns[a]));
  for (const auto& kv : classes) {
    const int s = tqr_autotune_run(kv.second.first, kv.second.second, stream);
    if (s != TQR_OK) return s;
  }
  std::map<std::pair<int, int>, TuneEntry> measured;
  {
    std::lock_guard<std::mutex> lk(g_tmu);
    measured = g_table;
  }
  constexpr int kPolicies = 5;
  auto policy = [&](int pol, int64_t m, int64_t n, int* nb, int* ib) {
    rule_tiles(m, n, nb, ib);
    if (pol == 1) {
      *ib = std::min(8, *nb);
      return;
    }
    if (pol == 0) return;
    auto it = measured.find(tune_class(m, n));
    if (it == measured.end()) return;
    if (pol == 4 && std::max(m, n) > 512) return;
    *nb = it->second.nb;
    *ib = it->second.ib;
    if (pol == 3 && *nb % 16 == 0) *ib = 16;
  };
  // one allocation for every matrix and the largest T of any policy
  std::vector<size_t> aoff(count), toff(count);
  size_t abytes = 0, tbytes = 0;
  for (int a = 0; a < count; ++a) {
    aoff[a] = abytes;
    abytes += ((sizeof(double) * static_cast<size_t>(ms[a]) * ns[a]) + 255) & ~size_t(255);
    size_t tmax = 0;
    for (int pol = 0; pol < kPolicies; ++pol) {
      int nb, ib;
      policy(pol, ms[a], ns[a], &nb, &ib);
      tmax = std::max(tmax, tqr_t_size(ms[a], ns[a], nb, ib));
    }
    toff[a] = tbytes;
    tbytes += (tmax + 255) & ~size_t(255);
  }
  char* buf = nullptr;
  if (lib_malloc(reinterpret_cast<void**>(&buf), abytes + tbytes, st) != cudaSuccess) {
    cudaGetLastError();
    return TQR_ERR_NOMEM;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  std::vector<tqr_desc> d(count);
  int best = 0, status = TQR_OK;
  float best_ms = INFINITY;
  for (int pol = 0; pol < kPolicies && status == TQR_OK; ++pol) {
    for (int a = 0; a < count; ++a) {
      int nb, ib;
      policy(pol, ms[a], ns[a], &nb, &ib);
      d[a].m = ms[a];
      d[a].n = ns[a];
      d[a].A = reinterpret_cast<double*>(buf + aoff[a]);
      d[a].lda = ms[a];
      d[a].T = reinterpret_cast<double*>(buf + abytes + toff[a]);
      d[a].nb = nb;
      d[a].ib = ib;
    }
    float ms_best = INFINITY;
    for (int rep = 0; rep < 2; ++rep) {  // the first builds the plan and graph
      tune_fill<<<4096, 256, 0, st>>>(reinterpret_cast<double*>(buf), static_cast<long long>(abytes / 8));
      uint64_t ticket = 0;
      cudaEventRecord(e0, st);
      int s = tqr_batch_submit(count, d.data(), &ticket, st);
      if (s == TQR_OK) s = tqr_batch_wait(ticket, nullptr);
      cudaEventRecord(e1, st);
      if (s != TQR_OK || cudaEventSynchronize(e1) != cudaSuccess) {
        status = s != TQR_OK ? s : TQR_ERR_CUDA;
        break;
      }
      float t = 0.0f;
      cudaEventElapsedTime(&t, e0, e1);
      if (rep > 0) ms_best = t;
    }
    if (status == TQR_OK && ms_best < best_ms) {
      best_ms = ms_best;
      best = pol;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(buf, st);
  cudaStreamSynchronize(st);
  if (status != TQR_OK) return status;
  // the winning policy's choice for every class of the batch
  std::lock_guard<std::mutex> lk(g_tmu);
  for (const auto& kv : classes) {
    int nb, ib;
    policy(best, kv.second.first, kv.second.second, &nb, &ib);
    g_table[kv.first] = {nb, ib, best_ms * 1e3 / count};
  }
  return TQR_OK;
}

extern "C" int tqr_autotune_save(const char* path) {
  if (path == nullptr) return -1;
  FILE* f = std::fopen(path, "w");
  if (!f) return TQR_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lk(g_tmu);
  std::fprintf(f, "# tqr autotune table: ceil(log2 m) ceil(log2 n) nb ib us_per_matrix\n");
  for (const auto& kv : g_table)
    std::fprintf(f, "%d %d %d %d %.6g\n", kv.first.first, kv.first.second, kv.second.nb, kv.second.ib,
                 kv.second.us_per_matrix);
  std::fclose(f);
  return TQR_OK;
}

extern "C" int tqr_autotune_load(const char* path) {
  if (path == nullptr) return -1;
  FILE* f = std::fopen(path, "r");
  if (!f) return TQR_ERR_UNSUPPORTED;
  char line[256];
  int status = TQR_OK;
  std::vector<std::pair<std::pair<int, int>, TuneEntry>> got;
  while (std::fgets(line, sizeof(line), f)) {
    if (line[0] == '#' || line[0] == '\n') continue;
    int a, b, nb, ib;
    double us;
    if (std::sscanf(line, "%d %d %d %d %lf", &a, &b, &nb, &ib, &us) != 5 || nb < 8 || nb > 256 || nb % 8 != 0 ||
        ib < 1 || ib > 64 || nb % ib != 0 || a < 0 || a > 40 || b < 0 || b > 40) {
      status = TQR_ERR_UNSUPPORTED;
      break;
    }
    got.push_back({{a, b}, {nb, ib, us}});
  }
  std::fclose(f);
  if (status != TQR_OK) return status;
  std::lock_guard<std::mutex> lk(g_tmu);
  for (const auto& kv : got) g_table[kv.first] = kv.second;
  return TQR_OK;
}

extern "C" int tqr_autotune_clear(void) {
  std::lock_guard<std::mutex> lk(g_tmu);
  g_table.clear();
  return TQR_OK;
}

// Host-only hooks for the tests: the class of a shape, and a table entry put
// by hand (the selection and the file format need no GPU).
extern "C" int tqr_debug_autotune_class(int64_t m, int64_t n, int* mb, int* nbin) {
  if (mb == nullptr || nbin == nullptr) return -3;
  const auto c = tune_class(m, n);
  *mb = c.first;
  *nbin = c.second;
  return TQR_OK;
}

extern "C" int tqr_debug_autotune_put(int64_t m, int64_t n, int nb, int ib, double us) {
  if (nb < 8 || nb > 256 || nb % 8 != 0 || ib < 1 || ib > 64 || nb % ib != 0) return -3;
  std::lock_guard<std::mutex> lk(g_tmu);
  g_table[tune_class(m, n)] = {nb, ib, us};
  return TQR_OK;
}
