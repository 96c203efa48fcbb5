// qsvm_api.cu -- host side of the C ABI declared in include/qsvm.h: argument
// checks, size queries, tile bookkeeping and kernel dispatch.  No allocation.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>

#include "qsvm_common.cuh"

#include <atomic>
#include <mutex>
#include <vector>

namespace qsvm {
cudaError_t launch_build_mps(const double* X, int64_t N, int n, int reps, int prec, void* mps, cudaStream_t st);
cudaError_t launch_pair(int chi, int prec, const TileArgs& a, int64_t ntiles, const PipeCfg& pc, cudaStream_t st);
cudaError_t prepare_persistent(int chi, int prec, const PipeCfg& pc, int64_t total_tiles, int* grid_out);
cudaError_t launch_persistent(int chi, int prec, const BatchArgs& a, const PipeCfg& pc, int grid, cudaStream_t st);
int pair_tile_dim(int chi, int prec);
int pair_threads(int chi, int prec);
cudaError_t pair_status(cudaStream_t st, int clear, int32_t* out);
int num_pipe_shapes();
cudaError_t launch_wait_timeout_selftest(uint64_t limit_ns, cudaStream_t st);
cudaError_t launch_sv_gram(const double* X, int64_t N, int n, int reps, void* ws, double* K, int64_t ldk,
                           cudaStream_t st);
struct DevSvcProblem {
  const int64_t* idx;
  const int8_t* y;
  int64_t n;
  double* alpha;
  double* g;
};
cudaError_t launch_svc_fit(const double* K, int64_t ldk, const DevSvcProblem* probs, int n_probs, double C, double tol,
                           int64_t max_iter, double* b_out, int64_t* iters_out, cudaStream_t st);
cudaError_t launch_svc_decision(const double* Kx, int64_t ldk, int64_t m, const DevSvcProblem* probs, int n_probs,
                                const double* b, double* F, cudaStream_t st);
PipeCfg make_pipe(int chi, int prec, int config);
PipeCfg whole_tile_pipe(int chi, int prec, int config);
int pipe_smem(const PipeCfg& pc, int chi, int prec);
}  // namespace qsvm

using namespace qsvm;

namespace {

thread_local std::string g_last_error;

int32_t fail(int32_t code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

int32_t cuda_fail(cudaError_t e, const char* where) {
  return fail(QSVM_ERR_CUDA, "%s: %s (%s)", where, cudaGetErrorName(e), cudaGetErrorString(e));
}

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

int32_t check_common(int32_t n_qubits, int32_t reps, int32_t precision) {
  if (reps < 1 || reps > 3) return fail(QSVM_ERR_CHI, "reps=%d: chi = 2^reps must be 2, 4 or 8", reps);
  if (n_qubits < 2) return fail(QSVM_ERR_ARG, "n_qubits=%d: the chain needs at least 2 qubits", n_qubits);
  if (precision < QSVM_FP64 || precision > QSVM_FP32_SPLIT)
    return fail(QSVM_ERR_ARG, "precision=%d is not a qsvm_precision", precision);
  return QSVM_OK;
}

int64_t tiles_per_side(int64_t n_points, int tdim) { return (n_points + tdim - 1) / tdim; }

// byte offset of the column-side (b-form) records inside an MPS buffer
size_t form_b_offset(int64_t n_points, int n_qubits, int reps, int prec) {
  const int chi = 1 << reps;
  return record_forms(chi, prec) == 2
             ? record_bytes(chi, prec) * (size_t)n_points * (size_t)record_sites(n_qubits, chi, prec)
             : 0;
}

// selected pipeline configuration per (reps - 1, precision); -1 = default
std::atomic<int> g_config[3][3] = {{{-1}, {-1}, {-1}}, {{-1}, {-1}, {-1}}, {{-1}, {-1}, {-1}}};

PipeCfg current_pipe(int reps, int prec) { return make_pipe(1 << reps, prec, g_config[reps - 1][prec].load()); }
// the batch (persistent) kernel: the selected shape, always whole tiles per CTA
PipeCfg current_batch_pipe(int reps, int prec) {
  return whole_tile_pipe(1 << reps, prec, g_config[reps - 1][prec].load());
}

constexpr int kMaxSmemPerCta = 227 * 1024;

// pairs contracted by upper-triangle tile (ti, tj) of a T x T grid over n_points
int64_t tile_pairs(int64_t ti, int64_t tj, int64_t n_points, int tdim) {
  const int64_t ni = std::min<int64_t>(tdim, n_points - ti * tdim);
  const int64_t nj = std::min<int64_t>(tdim, n_points - tj * tdim);
  return (ti == tj) ? ni * (ni + 1) / 2 : ni * nj;
}

int32_t gram_launch(const void* mps, int64_t n_points, int32_t n_qubits, int32_t reps, int32_t precision,
                    int64_t tile_begin, int64_t tile_end, double* K, int64_t ldk, double* logK, int64_t ldl,
                    void* stream) {
  int32_t rc = check_common(n_qubits, reps, precision);
  if (rc) return rc;
  if (n_points < 1) return fail(QSVM_ERR_ARG, "n_points=%lld must be >= 1", (long long)n_points);
  if (!mps || !aligned(mps, 16)) return fail(QSVM_ERR_ARG, "mps must be a non-null 16-byte aligned device pointer");
  if (!K || !aligned(K, 8)) return fail(QSVM_ERR_ARG, "K must be a non-null 8-byte aligned device pointer");
  if (ldk < n_points) return fail(QSVM_ERR_ARG, "ldk=%lld < n_points=%lld", (long long)ldk, (long long)n_points);
  if (logK && (!aligned(logK, 8) || ldl < n_points))
    return fail(QSVM_ERR_ARG, "logK must be 8-byte aligned with ldl >= n_points");
  const int chi = 1 << reps;
  const int tdim = pair_tile_dim(chi, precision);
  const int64_t T = tiles_per_side(n_points, tdim);
  const int64_t total = T * (T + 1) / 2;
  if (tile_begin < 0 || tile_end > total || tile_begin > tile_end)
    return fail(QSVM_ERR_ARG, "tile range [%lld, %lld) outside [0, %lld)", (long long)tile_begin,
                (long long)tile_end, (long long)total);
  if (tile_begin == tile_end) return QSVM_OK;
  TileArgs a{};
  a.mpsA = static_cast<const uint8_t*>(mps);
  a.mpsB = a.mpsA + form_b_offset(n_points, n_qubits, reps, precision);
  a.nA = a.nB = n_points;
  a.n = n_qubits;
  a.symmetric = 1;
  a.tile_begin = tile_begin;
  a.tiles_j = T;
  a.K = K;
  a.ldk = ldk;
  a.logK = logK;
  a.ldl = ldl;
  cudaError_t e = launch_pair(chi, precision, a, tile_end - tile_begin, current_pipe(reps, precision),
                              static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "pair kernel launch");
  return QSVM_OK;
}

// ---- batch job table -------------------------------------------------------
constexpr size_t kWsAlign = 256;
constexpr size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }
constexpr size_t ws_jobs_offset() { return kWsAlign; }
constexpr size_t ws_prefix_offset(int n_jobs) {
  return align_up(ws_jobs_offset() + sizeof(DevJob) * (size_t)n_jobs, kWsAlign);
}
constexpr size_t ws_total(int n_jobs) {
  return align_up(ws_prefix_offset(n_jobs) + sizeof(int64_t) * (size_t)(n_jobs + 1), kWsAlign);
}

// Host image of the workspace (counter slot, sorted job table, tile prefix).
struct BatchImage {
  std::vector<uint8_t> bytes;
  int64_t total_tiles = 0;
};

int32_t build_batch_image(const qsvm_job* jobs, int32_t n_jobs, int32_t reps, int32_t precision, const void* ws,
                          size_t ws_bytes, BatchImage& img) {
  int32_t rc = check_common(2, reps, precision);
  if (rc) return rc;
  if (!jobs || n_jobs < 1) return fail(QSVM_ERR_ARG, "jobs must be a non-empty host array");
  if (!ws || !aligned(ws, kWsAlign)) return fail(QSVM_ERR_ARG, "ws must be a non-null 256-byte aligned device pointer");
  if (ws_bytes < ws_total(n_jobs))
    return fail(QSVM_ERR_WORKSPACE, "ws_bytes=%zu < required %zu", ws_bytes, ws_total(n_jobs));
  const int tdim = pair_tile_dim(1 << reps, precision);
  std::vector<int> order((size_t)n_jobs);
  for (int j = 0; j < n_jobs; ++j) {
    const qsvm_job& J = jobs[j];
    if (!J.mps || !aligned(J.mps, 16) || J.n_points < 1 || J.n_qubits < 2 || !J.K || !aligned(J.K, 8) ||
        J.ldk < J.n_points || (J.logK && (!aligned(J.logK, 8) || J.ldl < J.n_points)) || J.reserved != 0)
      return fail(QSVM_ERR_ARG, "job %d: invalid pointer, size or leading dimension", j);
    order[(size_t)j] = j;
  }
  // heaviest tiles first: cost per tile grows with the qubit count
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return jobs[a].n_qubits > jobs[b].n_qubits; });
  img.bytes.assign(ws_total(n_jobs), 0);
  DevJob* dj = reinterpret_cast<DevJob*>(img.bytes.data() + ws_jobs_offset());
  int64_t* prefix = reinterpret_cast<int64_t*>(img.bytes.data() + ws_prefix_offset(n_jobs));
  int64_t acc = 0;
  for (int k = 0; k < n_jobs; ++k) {
    const qsvm_job& J = jobs[order[(size_t)k]];
    const int64_t T = tiles_per_side(J.n_points, tdim);
    dj[k].mps = static_cast<const uint8_t*>(J.mps);
    dj[k].n_points = J.n_points;
    dj[k].tiles = T;
    dj[k].K = J.K;
    dj[k].ldk = J.ldk;
    dj[k].logK = J.logK;
    dj[k].ldl = J.ldl;
    dj[k].n_qubits = J.n_qubits;
    dj[k].pad = 0;
    prefix[k] = acc;
    acc += T * (T + 1) / 2;
  }
  prefix[n_jobs] = acc;
  img.total_tiles = acc;
  return QSVM_OK;
}

BatchArgs batch_args(void* ws, int32_t n_jobs, int64_t total) {
  BatchArgs a{};
  uint8_t* base = static_cast<uint8_t*>(ws);
  a.counter = reinterpret_cast<unsigned long long*>(base);
  a.jobs = reinterpret_cast<const DevJob*>(base + ws_jobs_offset());
  a.prefix = reinterpret_cast<const int64_t*>(base + ws_prefix_offset(n_jobs));
  a.n_jobs = n_jobs;
  a.total_tiles = total;
  return a;
}

}  // namespace

struct qsvm_batch_plan {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int device = 0;
};

extern "C" {

size_t qsvm_mps_record_bytes(int32_t reps, int32_t precision) {
  if (reps < 1 || reps > 3 || precision < QSVM_FP64 || precision > QSVM_FP32_SPLIT) return 0;
  return record_bytes(1 << reps, precision);
}

size_t qsvm_mps_point_bytes(int32_t n_qubits, int32_t reps, int32_t precision) {
  if (n_qubits < 1) return 0;
  const size_t rec = qsvm_mps_record_bytes(reps, precision);
  return rec ? rec * (size_t)record_sites(n_qubits, 1 << reps, precision) : 0;
}

size_t qsvm_mps_bytes(int32_t n_qubits, int32_t reps, int64_t n_points, int32_t precision) {
  if (n_qubits < 1 || n_points < 0) return 0;
  return qsvm_mps_point_bytes(n_qubits, reps, precision) * (size_t)record_forms(1 << reps, precision) *
         (size_t)n_points;
}

int32_t qsvm_build_mps(const double* X, int64_t n_points, int32_t n_qubits, int32_t reps, int32_t precision,
                       void* mps, size_t mps_bytes, void* stream) {
  int32_t rc = check_common(n_qubits, reps, precision);
  if (rc) return rc;
  if (n_points < 1) return fail(QSVM_ERR_ARG, "n_points=%lld must be >= 1", (long long)n_points);
  if (!X || !aligned(X, 8)) return fail(QSVM_ERR_ARG, "X must be a non-null 8-byte aligned device pointer");
  if (!mps || !aligned(mps, 16)) return fail(QSVM_ERR_ARG, "mps must be a non-null 16-byte aligned device pointer");
  const size_t need = qsvm_mps_bytes(n_qubits, reps, n_points, precision);
  if (mps_bytes < need)
    return fail(QSVM_ERR_ARG, "mps_bytes=%zu < required %zu", mps_bytes, need);
  cudaError_t e = launch_build_mps(X, n_points, n_qubits, reps, precision, mps, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "build_mps launch");
  return QSVM_OK;
}

int32_t qsvm_gram_tile_dim(int32_t reps, int32_t precision) {
  if (reps < 1 || reps > 3 || precision < QSVM_FP64 || precision > QSVM_FP32_SPLIT) return 0;
  return pair_tile_dim(1 << reps, precision);
}

int64_t qsvm_gram_num_tiles(int64_t n_points, int32_t reps, int32_t precision) {
  const int tdim = qsvm_gram_tile_dim(reps, precision);
  if (tdim <= 0 || n_points < 1) return 0;
  const int64_t T = tiles_per_side(n_points, tdim);
  return T * (T + 1) / 2;
}

int32_t qsvm_gram_partition(int64_t n_points, int32_t reps, int32_t precision, int32_t world, int32_t rank,
                            int64_t* tile_begin, int64_t* tile_end) {
  if (!tile_begin || !tile_end) return fail(QSVM_ERR_ARG, "null output pointer");
  if (world < 1 || rank < 0 || rank >= world) return fail(QSVM_ERR_ARG, "rank %d of world %d", rank, world);
  const int tdim = qsvm_gram_tile_dim(reps, precision);
  if (tdim <= 0) return fail(QSVM_ERR_CHI, "reps=%d precision=%d not supported", reps, precision);
  if (n_points < 1) return fail(QSVM_ERR_ARG, "n_points=%lld must be >= 1", (long long)n_points);
  const int64_t T = tiles_per_side(n_points, tdim);
  const int64_t total_tiles = T * (T + 1) / 2;
  const int64_t total_pairs = n_points * (n_points + 1) / 2;
  // boundary r sits at the first tile (in tile order) whose prefix pair count
  // reaches r/world of the total (tiles are whole, so shares differ by at most one tile)
  auto boundary = [&](int64_t r) -> int64_t {
    if (r <= 0) return 0;
    if (r >= world) return total_tiles;
    const double target = (double)total_pairs * (double)r / (double)world;
    double acc = 0;
    for (int64_t b = 0; b < total_tiles; ++b) {
      if (acc >= target) return b;
      int64_t ti, tj;
      sym_tile_decode(b, T, ti, tj);
      acc += (double)tile_pairs(ti, tj, n_points, tdim);
    }
    return total_tiles;
  };
  *tile_begin = boundary(rank);
  *tile_end = boundary(rank + 1);
  return QSVM_OK;
}

int32_t qsvm_gram_tile_coords(int64_t n_points, int32_t reps, int32_t precision, int64_t tile, int64_t* ti,
                              int64_t* tj) {
  if (!ti || !tj) return fail(QSVM_ERR_ARG, "null output pointer");
  const int64_t total = qsvm_gram_num_tiles(n_points, reps, precision);
  if (total <= 0) return fail(QSVM_ERR_ARG, "no tiles for n_points=%lld reps=%d precision=%d", (long long)n_points,
                              reps, precision);
  if (tile < 0 || tile >= total) return fail(QSVM_ERR_ARG, "tile %lld outside [0, %lld)", (long long)tile, (long long)total);
  sym_tile_decode(tile, tiles_per_side(n_points, qsvm_gram_tile_dim(reps, precision)), *ti, *tj);
  return QSVM_OK;
}

int32_t qsvm_gram_tile_list(int64_t n_points, int32_t reps, int32_t precision, int64_t tile_begin,
                            int64_t tile_end, int64_t* ti, int64_t* tj) {
  const int64_t total = qsvm_gram_num_tiles(n_points, reps, precision);
  if (total <= 0) return fail(QSVM_ERR_ARG, "no tiles for n_points=%lld reps=%d precision=%d", (long long)n_points,
                              reps, precision);
  if (tile_begin < 0 || tile_end < tile_begin || tile_end > total)
    return fail(QSVM_ERR_ARG, "tile range [%lld, %lld) outside [0, %lld]", (long long)tile_begin,
                (long long)tile_end, (long long)total);
  if (tile_end > tile_begin && (!ti || !tj)) return fail(QSVM_ERR_ARG, "null output pointer");
  const int64_t T = tiles_per_side(n_points, qsvm_gram_tile_dim(reps, precision));
  for (int64_t b = tile_begin; b < tile_end; ++b) sym_tile_decode(b, T, ti[b - tile_begin], tj[b - tile_begin]);
  return QSVM_OK;
}

int32_t qsvm_kernel_gram_tiles(const void* mps, int64_t n_points, int32_t n_qubits, int32_t reps,
                               int32_t precision, int64_t tile_begin, int64_t tile_end, double* K, int64_t ldk,
                               double* logK, int64_t ldl, void* stream) {
  return gram_launch(mps, n_points, n_qubits, reps, precision, tile_begin, tile_end, K, ldk, logK, ldl, stream);
}

int32_t qsvm_kernel_gram(const void* mps, int64_t n_points, int32_t n_qubits, int32_t reps, int32_t precision,
                         double* K, int64_t ldk, double* logK, int64_t ldl, void* stream) {
  const int64_t total = qsvm_gram_num_tiles(n_points, reps, precision);
  return gram_launch(mps, n_points, n_qubits, reps, precision, 0, total, K, ldk, logK, ldl, stream);
}

int32_t qsvm_kernel_cross(const void* mps_a, int64_t n_a, const void* mps_b, int64_t n_b, int32_t n_qubits,
                          int32_t reps, int32_t precision, double* K, int64_t ldk, double* logK, int64_t ldl,
                          void* stream) {
  int32_t rc = check_common(n_qubits, reps, precision);
  if (rc) return rc;
  if (n_a < 1 || n_b < 1) return fail(QSVM_ERR_ARG, "n_a=%lld, n_b=%lld must be >= 1", (long long)n_a, (long long)n_b);
  if (!mps_a || !mps_b || !aligned(mps_a, 16) || !aligned(mps_b, 16))
    return fail(QSVM_ERR_ARG, "mps_a and mps_b must be non-null 16-byte aligned device pointers");
  if (!K || !aligned(K, 8)) return fail(QSVM_ERR_ARG, "K must be a non-null 8-byte aligned device pointer");
  if (ldk < n_b) return fail(QSVM_ERR_ARG, "ldk=%lld < n_b=%lld", (long long)ldk, (long long)n_b);
  if (logK && (!aligned(logK, 8) || ldl < n_b)) return fail(QSVM_ERR_ARG, "logK must be 8-byte aligned with ldl >= n_b");
  const int chi = 1 << reps;
  const int tdim = pair_tile_dim(chi, precision);
  const int64_t Ta = tiles_per_side(n_a, tdim), Tb = tiles_per_side(n_b, tdim);
  TileArgs a{};
  a.mpsA = static_cast<const uint8_t*>(mps_a);
  a.mpsB = static_cast<const uint8_t*>(mps_b) + form_b_offset(n_b, n_qubits, reps, precision);
  a.nA = n_a;
  a.nB = n_b;
  a.n = n_qubits;
  a.symmetric = 0;
  a.tile_begin = 0;
  a.tiles_i = Ta;
  a.tiles_j = Tb;
  a.K = K;
  a.ldk = ldk;
  a.logK = logK;
  a.ldl = ldl;
  cudaError_t e = launch_pair(chi, precision, a, Ta * Tb, current_pipe(reps, precision), static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "pair kernel launch");
  return QSVM_OK;
}

// ---- Gram of host data ------------------------------------------------------
// Device scratch of qsvm_gram_host: X, the MPS, K (and logK), each 256-byte aligned.
static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Number of chunks a host-buffer call splits its launches into: at most kMaxChunks,
// and at least 4 CTAs (one per tile) per SM in each, so small problems run as one
// launch instead of several that each leave most SMs idle.
constexpr int kMaxChunks = 8;
static int host_chunks(int64_t tiles) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                               cudaSuccess || sms < 1)
    sms = 1;
  const int64_t c = tiles / (4 * (int64_t)sms);
  return (int)std::max<int64_t>(1, std::min<int64_t>(kMaxChunks, c));
}

size_t qsvm_gram_host_workspace_bytes(int64_t n_points, int32_t n_qubits, int32_t reps, int32_t precision,
                                      int32_t with_logk) {
  if (n_points < 1 || n_qubits < 2) return 0;
  const size_t mps = qsvm_mps_bytes(n_qubits, reps, n_points, precision);
  if (mps == 0) return 0;
  const size_t k = align256((size_t)n_points * (size_t)n_points * sizeof(double));
  return align256((size_t)n_points * (size_t)n_qubits * sizeof(double)) + align256(mps) + k * (with_logk ? 2 : 1);
}

int32_t qsvm_gram_host(const double* X, int64_t n_points, int32_t n_qubits, int32_t reps, int32_t precision,
                       double* K, int64_t ldk, double* logK, int64_t ldl, void* ws, size_t ws_bytes, void* stream) {
  int32_t rc = check_common(n_qubits, reps, precision);
  if (rc) return rc;
  if (n_points < 1) return fail(QSVM_ERR_ARG, "n_points=%lld must be >= 1", (long long)n_points);
  if (!X || !K) return fail(QSVM_ERR_ARG, "X and K must be non-null host pointers");
  if (ldk < n_points) return fail(QSVM_ERR_ARG, "ldk=%lld < n_points=%lld", (long long)ldk, (long long)n_points);
  if (logK && ldl < n_points) return fail(QSVM_ERR_ARG, "ldl=%lld < n_points=%lld", (long long)ldl, (long long)n_points);
  const size_t need = qsvm_gram_host_workspace_bytes(n_points, n_qubits, reps, precision, logK != nullptr);
  if (!ws || !aligned(ws, 256)) return fail(QSVM_ERR_ARG, "ws must be a non-null 256-byte aligned device pointer");
  if (ws_bytes < need) return fail(QSVM_ERR_ARG, "ws_bytes=%zu < required %zu", ws_bytes, need);
  const int64_t N = n_points;
  uint8_t* base = static_cast<uint8_t*>(ws);
  double* dX = reinterpret_cast<double*>(base);
  base += align256((size_t)N * (size_t)n_qubits * sizeof(double));
  void* dM = base;
  const size_t mps_bytes = qsvm_mps_bytes(n_qubits, reps, N, precision);
  base += align256(mps_bytes);
  double* dK = reinterpret_cast<double*>(base);
  double* dL = logK ? reinterpret_cast<double*>(base + align256((size_t)N * (size_t)N * sizeof(double))) : nullptr;
  cudaStream_t st = static_cast<cudaStream_t>(stream);

  cudaError_t e = cudaMemcpyAsync(dX, X, (size_t)N * (size_t)n_qubits * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e, "copy of X to the device");
  rc = qsvm_build_mps(dX, N, n_qubits, reps, precision, dM, mps_bytes, stream);
  if (rc) return rc;

  // Chunks of whole tile bands, up to kMaxChunks of them by tile count.  Bands run in
  // order and a band's rows receive mirror writes only from earlier bands, so the
  // rows of chunk c are final once chunks 0..c have completed: a copy stream, which
  // waits for each chunk in turn, copies them out while later chunks compute.  The
  // chunks write disjoint tiles, so consecutive chunks alternate between the caller's
  // stream and a second compute stream: a launch fills the SMs its predecessor's last
  // wave leaves idle.
  constexpr int kChunks = kMaxChunks;
  const int tdim = pair_tile_dim(1 << reps, precision);
  const int64_t T = tiles_per_side(N, tdim);
  const int64_t total = T * (T + 1) / 2;
  const int64_t nbands = (T + kBandRows - 1) / kBandRows;
  const int nch = host_chunks(total);
  auto band_start = [&](int64_t b) { return b >= nbands ? total : sym_band_start(b, T); };
  cudaStream_t cs = nullptr, xs = nullptr;  // second compute stream, copy stream
  cudaEvent_t ev[kChunks + 3] = {};         // chunks, build, joins of cs and xs
  e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&xs, cudaStreamNonBlocking);
  for (int c = 0; e == cudaSuccess && c < kChunks + 3; ++c) e = cudaEventCreateWithFlags(&ev[c], cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(ev[kChunks], st);  // the MPS is built
  if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ev[kChunks], 0);
  int64_t b0 = 0;
  for (int c = 0; e == cudaSuccess && rc == QSVM_OK && b0 < nbands; ++c) {
    int64_t b1 = b0 + 1;  // the last chunk takes every remaining band
    while (c < nch - 1 && b1 < nbands && band_start(b1) * nch < total * (int64_t)(c + 1)) ++b1;
    if (c == nch - 1) b1 = nbands;
    cudaStream_t run = (c & 1) ? cs : st;
    rc = gram_launch(dM, N, n_qubits, reps, precision, band_start(b0), band_start(b1), dK, N, dL, N, run);
    if (rc) break;
    const int64_t r0 = b0 * kBandRows * tdim, r1 = std::min<int64_t>(N, b1 * kBandRows * tdim);
    e = cudaEventRecord(ev[c], run);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(xs, ev[c], 0);
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(K + r0 * ldk, (size_t)ldk * sizeof(double), dK + r0 * N, (size_t)N * sizeof(double),
                            (size_t)N * sizeof(double), (size_t)(r1 - r0), cudaMemcpyDeviceToHost, xs);
    if (e == cudaSuccess && logK)
      e = cudaMemcpy2DAsync(logK + r0 * ldl, (size_t)ldl * sizeof(double), dL + r0 * N, (size_t)N * sizeof(double),
                            (size_t)N * sizeof(double), (size_t)(r1 - r0), cudaMemcpyDeviceToHost, xs);
    b0 = b1;
  }
  // join both helper streams back into the caller's stream (also after an error, so
  // that nothing of this call is left unordered), then release them (deferred)
  cudaError_t e2 = cudaSuccess;
  cudaStream_t helpers[2] = {cs, xs};
  for (int h = 0; h < 2; ++h) {
    if (!helpers[h] || !ev[kChunks + 1 + h]) continue;
    cudaError_t r = cudaEventRecord(ev[kChunks + 1 + h], helpers[h]);
    if (r == cudaSuccess) r = cudaStreamWaitEvent(st, ev[kChunks + 1 + h], 0);
    if (r != cudaSuccess && e2 == cudaSuccess) e2 = r;
  }
  for (auto& x : ev)
    if (x) cudaEventDestroy(x);
  if (cs) cudaStreamDestroy(cs);
  if (xs) cudaStreamDestroy(xs);
  if (rc) return rc;
  if (e != cudaSuccess) return cuda_fail(e, "chunked Gram or copy of K to the host");
  if (e2 != cudaSuccess) return cuda_fail(e2, "joining the helper streams");
  return QSVM_OK;
}

size_t qsvm_cross_host_workspace_bytes(int64_t n_a, int64_t n_b, int32_t n_qubits, int32_t reps, int32_t precision,
                                       int32_t with_logk) {
  if (n_a < 1 || n_b < 1 || n_qubits < 2) return 0;
  const size_t ma = qsvm_mps_bytes(n_qubits, reps, n_a, precision), mb = qsvm_mps_bytes(n_qubits, reps, n_b, precision);
  if (ma == 0 || mb == 0) return 0;
  const size_t k = align256((size_t)n_a * (size_t)n_b * sizeof(double));
  return align256((size_t)(n_a + n_b) * (size_t)n_qubits * sizeof(double)) + align256(ma) + align256(mb) +
         k * (with_logk ? 2 : 1);
}

int32_t qsvm_cross_host(const double* X_a, int64_t n_a, const double* X_b, int64_t n_b, int32_t n_qubits,
                        int32_t reps, int32_t precision, double* K, int64_t ldk, double* logK, int64_t ldl, void* ws,
                        size_t ws_bytes, void* stream) {
  int32_t rc = check_common(n_qubits, reps, precision);
  if (rc) return rc;
  if (n_a < 1 || n_b < 1) return fail(QSVM_ERR_ARG, "n_a=%lld, n_b=%lld must be >= 1", (long long)n_a, (long long)n_b);
  if (!X_a || !X_b || !K) return fail(QSVM_ERR_ARG, "X_a, X_b and K must be non-null host pointers");
  if (ldk < n_b) return fail(QSVM_ERR_ARG, "ldk=%lld < n_b=%lld", (long long)ldk, (long long)n_b);
  if (logK && ldl < n_b) return fail(QSVM_ERR_ARG, "ldl=%lld < n_b=%lld", (long long)ldl, (long long)n_b);
  const size_t need = qsvm_cross_host_workspace_bytes(n_a, n_b, n_qubits, reps, precision, logK != nullptr);
  if (!ws || !aligned(ws, 256)) return fail(QSVM_ERR_ARG, "ws must be a non-null 256-byte aligned device pointer");
  if (ws_bytes < need) return fail(QSVM_ERR_ARG, "ws_bytes=%zu < required %zu", ws_bytes, need);
  uint8_t* base = static_cast<uint8_t*>(ws);
  double* dXa = reinterpret_cast<double*>(base);
  double* dXb = dXa + (size_t)n_a * (size_t)n_qubits;
  base += align256((size_t)(n_a + n_b) * (size_t)n_qubits * sizeof(double));
  const size_t ma = qsvm_mps_bytes(n_qubits, reps, n_a, precision), mb = qsvm_mps_bytes(n_qubits, reps, n_b, precision);
  uint8_t* dMa = base;
  base += align256(ma);
  uint8_t* dMb = base;
  base += align256(mb);
  double* dK = reinterpret_cast<double*>(base);
  double* dL = logK ? reinterpret_cast<double*>(base + align256((size_t)n_a * (size_t)n_b * sizeof(double))) : nullptr;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(dXa, X_a, (size_t)n_a * (size_t)n_qubits * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dXb, X_b, (size_t)n_b * (size_t)n_qubits * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e, "copy of X_a, X_b to the device");
  rc = qsvm_build_mps(dXa, n_a, n_qubits, reps, precision, dMa, ma, stream);
  if (!rc) rc = qsvm_build_mps(dXb, n_b, n_qubits, reps, precision, dMb, mb, stream);
  if (rc) return rc;

  // Row chunks of whole tile rows, up to kMaxChunks of them: the rows of a chunk are
  // final when its launch completes, and a copy stream takes them to the host while
  // later chunks compute.  Chunks write disjoint rows, so they alternate between the
  // caller's stream and a second compute stream, as in qsvm_gram_host.
  constexpr int kChunks = kMaxChunks;
  const int tdim = pair_tile_dim(1 << reps, precision);
  const int64_t Ta = tiles_per_side(n_a, tdim), Tb = tiles_per_side(n_b, tdim);
  const int nch = host_chunks(Ta * Tb);
  const int64_t rows_per_chunk = ((Ta + nch - 1) / nch) * tdim;
  const size_t point_bytes = qsvm_mps_point_bytes(n_qubits, reps, precision);
  cudaStream_t cs = nullptr, xs = nullptr;  // second compute stream, copy stream
  cudaEvent_t ev[kChunks + 3] = {};         // chunks, build, joins of cs and xs
  e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&xs, cudaStreamNonBlocking);
  for (int c = 0; e == cudaSuccess && c < kChunks + 3; ++c) e = cudaEventCreateWithFlags(&ev[c], cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(ev[kChunks], st);  // both MPS are built
  if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ev[kChunks], 0);
  for (int c = 0; e == cudaSuccess && rc == QSVM_OK && c < nch; ++c) {
    const int64_t r0 = c * rows_per_chunk, r1 = std::min<int64_t>(n_a, r0 + rows_per_chunk);
    if (r0 >= r1) break;
    cudaStream_t run = (c & 1) ? cs : st;
    rc = qsvm_kernel_cross(dMa + (size_t)r0 * point_bytes, r1 - r0, dMb, n_b, n_qubits, reps, precision,
                           dK + r0 * n_b, n_b, dL ? dL + r0 * n_b : nullptr, n_b, run);
    if (rc) break;
    e = cudaEventRecord(ev[c], run);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(xs, ev[c], 0);
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(K + r0 * ldk, (size_t)ldk * sizeof(double), dK + r0 * n_b, (size_t)n_b * sizeof(double),
                            (size_t)n_b * sizeof(double), (size_t)(r1 - r0), cudaMemcpyDeviceToHost, xs);
    if (e == cudaSuccess && logK)
      e = cudaMemcpy2DAsync(logK + r0 * ldl, (size_t)ldl * sizeof(double), dL + r0 * n_b, (size_t)n_b * sizeof(double),
                            (size_t)n_b * sizeof(double), (size_t)(r1 - r0), cudaMemcpyDeviceToHost, xs);
  }
  // join both helper streams back into the caller's stream (also after an error), then
  // release them (deferred)
  cudaError_t e2 = cudaSuccess;
  cudaStream_t helpers[2] = {cs, xs};
  for (int h = 0; h < 2; ++h) {
    if (!helpers[h] || !ev[kChunks + 1 + h]) continue;
    cudaError_t r = cudaEventRecord(ev[kChunks + 1 + h], helpers[h]);
    if (r == cudaSuccess) r = cudaStreamWaitEvent(st, ev[kChunks + 1 + h], 0);
    if (r != cudaSuccess && e2 == cudaSuccess) e2 = r;
  }
  for (auto& x : ev)
    if (x) cudaEventDestroy(x);
  for (auto h : helpers)
    if (h) cudaStreamDestroy(h);
  if (rc) return rc;
  if (e != cudaSuccess) return cuda_fail(e, "chunked copy of the cross kernel to the host");
  if (e2 != cudaSuccess) return cuda_fail(e2, "joining the helper streams");
  return QSVM_OK;
}

size_t qsvm_batch_workspace_bytes(int32_t n_jobs) { return n_jobs < 1 ? 0 : ws_total(n_jobs); }

int32_t qsvm_kernel_batch(const qsvm_job* jobs, int32_t n_jobs, int32_t reps, int32_t precision, void* ws,
                          size_t ws_bytes, void* stream) {
  BatchImage img;
  int32_t rc = build_batch_image(jobs, n_jobs, reps, precision, ws, ws_bytes, img);
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // pageable source: the call returns once the bytes are staged, so img may go
  cudaError_t e = cudaMemcpyAsync(ws, img.bytes.data(), img.bytes.size(), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e, "batch job table upload");
  const BatchArgs a = batch_args(ws, n_jobs, img.total_tiles);
  const PipeCfg pc = current_batch_pipe(reps, precision);
  int grid = 0;
  e = prepare_persistent(1 << reps, precision, pc, img.total_tiles, &grid);
  if (e == cudaSuccess) e = launch_persistent(1 << reps, precision, a, pc, grid, st);
  if (e != cudaSuccess) return cuda_fail(e, "persistent kernel launch");
  return QSVM_OK;
}

int32_t qsvm_batch_plan_create(const qsvm_job* jobs, int32_t n_jobs, int32_t reps, int32_t precision, void* ws,
                               size_t ws_bytes, qsvm_batch_plan** plan_out) {
  if (!plan_out) return fail(QSVM_ERR_ARG, "plan_out is null");
  *plan_out = nullptr;
  BatchImage img;
  int32_t rc = build_batch_image(jobs, n_jobs, reps, precision, ws, ws_bytes, img);
  if (rc) return rc;
  cudaError_t e = cudaMemcpy(ws, img.bytes.data(), img.bytes.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "batch job table upload");
  auto* plan = new qsvm_batch_plan();
  cudaGetDevice(&plan->device);
  cudaStream_t cap = nullptr;
  e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    delete plan;
    return cuda_fail(e, "capture stream");
  }
  const BatchArgs a = batch_args(ws, n_jobs, img.total_tiles);
  const PipeCfg pc = current_batch_pipe(reps, precision);
  int grid = 0;
  e = prepare_persistent(1 << reps, precision, pc, img.total_tiles, &grid);
  if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaError_t e1 = cudaMemsetAsync(a.counter, 0, sizeof(unsigned long long), cap);
    cudaError_t e2 = (e1 == cudaSuccess) ? launch_persistent(1 << reps, precision, a, pc, grid, cap) : e1;
    e = cudaStreamEndCapture(cap, &plan->graph);
    if (e2 != cudaSuccess) e = e2;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&plan->exec, plan->graph, 0);
  cudaStreamDestroy(cap);
  if (e != cudaSuccess) {
    if (plan->graph) cudaGraphDestroy(plan->graph);
    delete plan;
    return cuda_fail(e, "batch graph capture");
  }
  *plan_out = plan;
  return QSVM_OK;
}

int32_t qsvm_batch_plan_launch(qsvm_batch_plan* plan, void* stream) {
  if (!plan || !plan->exec) return fail(QSVM_ERR_ARG, "null plan");
  cudaError_t e = cudaGraphLaunch(plan->exec, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "graph launch");
  return QSVM_OK;
}

int32_t qsvm_batch_plan_destroy(qsvm_batch_plan* plan) {
  if (!plan) return QSVM_OK;
  if (plan->exec) cudaGraphExecDestroy(plan->exec);
  if (plan->graph) cudaGraphDestroy(plan->graph);
  delete plan;
  return QSVM_OK;
}

int32_t qsvm_num_configs(void) { return num_pipe_shapes(); }

int32_t qsvm_config_info(int32_t index, int32_t reps, int32_t precision, int32_t* sites_per_chunk, int32_t* stages) {
  int32_t rc = check_common(2, reps, precision);
  if (rc) return rc;
  if (index < 0 || index >= num_pipe_shapes()) return fail(QSVM_ERR_ARG, "config index %d out of range", index);
  const PipeCfg pc = make_pipe(1 << reps, precision, index);
  if (sites_per_chunk) *sites_per_chunk = pc.S;
  if (stages) *stages = pc.stages;
  return QSVM_OK;
}

int32_t qsvm_config_tile(int32_t index, int32_t reps, int32_t precision, int32_t* pairs_per_side,
                         int32_t* threads_per_pair_out) {
  int32_t rc = check_common(2, reps, precision);
  if (rc) return rc;
  if (index < -1 || index >= num_pipe_shapes()) return fail(QSVM_ERR_ARG, "config index %d out of range", index);
  const PipeCfg pc = make_pipe(1 << reps, precision, index);
  if (pairs_per_side) *pairs_per_side = pc.tile;
  if (threads_per_pair_out) *threads_per_pair_out = pair_threads(1 << reps, precision);
  return QSVM_OK;
}

int32_t qsvm_set_config(int32_t reps, int32_t precision, int32_t index) {
  int32_t rc = check_common(2, reps, precision);
  if (rc) return rc;
  if (index < -1 || index >= num_pipe_shapes()) return fail(QSVM_ERR_ARG, "config index %d out of range", index);
  if (index >= 0 && pipe_smem(make_pipe(1 << reps, precision, index), 1 << reps, precision) > kMaxSmemPerCta)
    return fail(QSVM_ERR_ARG, "config %d needs more shared memory than a CTA has", index);
  g_config[reps - 1][precision].store(index);
  return QSVM_OK;
}

int32_t qsvm_get_config(int32_t reps, int32_t precision) {
  if (reps < 1 || reps > 3 || precision < QSVM_FP64 || precision > QSVM_FP32_SPLIT) return -1;
  return g_config[reps - 1][precision].load();
}

int32_t qsvm_autotune(const void* mps, int64_t n_points, int32_t n_qubits, int32_t reps, int32_t precision,
                      double* K, int64_t ldk, void* stream, int32_t* best_out, float* ms_out) {
  int32_t rc = check_common(n_qubits, reps, precision);
  if (rc) return rc;
  if (!best_out) return fail(QSVM_ERR_ARG, "best_out is null");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int prev = g_config[reps - 1][precision].load();
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) return cuda_fail(e, "event create");
  int best = -1;
  float best_ms = 0.f;
  int32_t out = QSVM_OK;
  for (int c = 0; c < num_pipe_shapes() && out == QSVM_OK; ++c) {
    float ms = -1.f;
    if (pipe_smem(make_pipe(1 << reps, precision, c), 1 << reps, precision) <= kMaxSmemPerCta) {
      g_config[reps - 1][precision].store(c);
      // one untimed run, then the timed one
      for (int it = 0; it < 2 && out == QSVM_OK; ++it) {
        if (it == 1) cudaEventRecord(e0, st);
        out = qsvm_kernel_gram(mps, n_points, n_qubits, reps, precision, K, ldk, nullptr, 0, stream);
        if (it == 1) cudaEventRecord(e1, st);
      }
      if (out == QSVM_OK) {
        e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) out = cuda_fail(e, "autotune timing");
        else cudaEventElapsedTime(&ms, e0, e1);
      }
      if (out == QSVM_OK && (best < 0 || ms < best_ms)) {
        best = c;
        best_ms = ms;
      }
    }
    if (ms_out) ms_out[c] = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  g_config[reps - 1][precision].store(out == QSVM_OK ? best : prev);
  if (out != QSVM_OK) return out;
  *best_out = best;
  return QSVM_OK;
}

int32_t qsvm_device_status(void* stream, int32_t clear, int32_t* status_out) {
  if (!status_out) return fail(QSVM_ERR_ARG, "status_out is null");
  int32_t v = 0;
  cudaError_t e = pair_status(static_cast<cudaStream_t>(stream), clear, &v);
  if (e != cudaSuccess) return cuda_fail(e, "reading the device status word");
  *status_out = v;
  return QSVM_OK;
}

size_t qsvm_sv_workspace_bytes(int64_t n_points, int32_t n_qubits) {
  if (n_points < 1 || n_qubits < 1 || n_qubits > 24) return 0;
  return (size_t)n_points * ((size_t)1 << n_qubits) * 16;
}

int32_t qsvm_sv_gram(const double* X, int64_t n_points, int32_t n_qubits, int32_t reps, double* K, int64_t ldk,
                     void* ws, size_t ws_bytes, void* stream) {
  if (n_qubits < 1 || n_qubits > 24) return fail(QSVM_ERR_ARG, "n_qubits=%d outside 1..24 for state vectors", n_qubits);
  if (reps < 1 || reps > 64) return fail(QSVM_ERR_ARG, "reps=%d outside 1..64", reps);
  if (n_points < 1) return fail(QSVM_ERR_ARG, "n_points=%lld must be >= 1", (long long)n_points);
  if (!X || !aligned(X, 8)) return fail(QSVM_ERR_ARG, "X must be a non-null 8-byte aligned device pointer");
  if (!K || !aligned(K, 8) || ldk < n_points) return fail(QSVM_ERR_ARG, "K must be 8-byte aligned with ldk >= n_points");
  if (!ws || !aligned(ws, 16)) return fail(QSVM_ERR_ARG, "ws must be a non-null 16-byte aligned device pointer");
  const size_t need = qsvm_sv_workspace_bytes(n_points, n_qubits);
  if (ws_bytes < need) return fail(QSVM_ERR_WORKSPACE, "ws_bytes=%zu < required %zu", ws_bytes, need);
  cudaError_t e = launch_sv_gram(X, n_points, n_qubits, reps, ws, K, ldk, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "state-vector launch");
  return QSVM_OK;
}

// ---- SVC on a precomputed kernel ----------------------------------------------
static size_t svc_table_bytes(int32_t n_problems) {
  return ((size_t)n_problems * sizeof(DevSvcProblem) + 255) / 256 * 256;
}

static int32_t svc_check(const qsvm_svc_problem* probs, int32_t n_problems) {
  if (!probs || n_problems < 1 || n_problems > 65535)
    return fail(QSVM_ERR_ARG, "problems must be a host array of 1..65535 entries");
  for (int32_t p = 0; p < n_problems; ++p) {
    const qsvm_svc_problem& P = probs[p];
    if (!P.idx || !aligned(P.idx, 8) || !P.y || !P.alpha || !aligned(P.alpha, 8) || P.n < 2)
      return fail(QSVM_ERR_ARG, "problem %d: null or misaligned pointer, or fewer than 2 points", p);
  }
  return QSVM_OK;
}

size_t qsvm_svc_workspace_bytes(const qsvm_svc_problem* problems, int32_t n_problems) {
  if (!problems || n_problems < 1) return 0;
  size_t g = 0;
  for (int32_t p = 0; p < n_problems; ++p) g += (size_t)(problems[p].n > 0 ? problems[p].n : 0);
  return svc_table_bytes(n_problems) + g * sizeof(double);
}

// writes the device problem table (and gradient slices) into ws on the stream
static int32_t svc_upload(const qsvm_svc_problem* probs, int32_t n_problems, void* ws, bool with_g, cudaStream_t st) {
  std::vector<DevSvcProblem> t((size_t)n_problems);
  double* g = reinterpret_cast<double*>(static_cast<uint8_t*>(ws) + svc_table_bytes(n_problems));
  for (int32_t p = 0; p < n_problems; ++p) {
    t[(size_t)p] = DevSvcProblem{probs[p].idx, probs[p].y, probs[p].n, probs[p].alpha, with_g ? g : nullptr};
    g += probs[p].n;
  }
  cudaError_t e = cudaMemcpyAsync(ws, t.data(), t.size() * sizeof(DevSvcProblem), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e, "svc problem table upload");
  return QSVM_OK;
}

int32_t qsvm_svc_fit(const double* K, int64_t ldk, const qsvm_svc_problem* problems, int32_t n_problems, double C,
                     double tol, int64_t max_iter, double* b_out, int64_t* iters_out, void* ws, size_t ws_bytes,
                     void* stream) {
  int32_t rc = svc_check(problems, n_problems);
  if (rc) return rc;
  if (!K || !aligned(K, 8) || ldk < 1) return fail(QSVM_ERR_ARG, "K must be a non-null 8-byte aligned device pointer");
  if (!(C > 0) || !(tol > 0) || max_iter < 1) return fail(QSVM_ERR_ARG, "C and tol must be > 0, max_iter >= 1");
  if (!b_out || !iters_out || !aligned(b_out, 8) || !aligned(iters_out, 8))
    return fail(QSVM_ERR_ARG, "b_out and iters_out must be 8-byte aligned device pointers");
  if (!ws || !aligned(ws, 256)) return fail(QSVM_ERR_ARG, "ws must be a non-null 256-byte aligned device pointer");
  if (ws_bytes < qsvm_svc_workspace_bytes(problems, n_problems))
    return fail(QSVM_ERR_WORKSPACE, "ws_bytes=%zu < required %zu", ws_bytes, qsvm_svc_workspace_bytes(problems, n_problems));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  rc = svc_upload(problems, n_problems, ws, true, st);
  if (rc) return rc;
  cudaError_t e = launch_svc_fit(K, ldk, static_cast<const DevSvcProblem*>(ws), n_problems, C, tol, max_iter, b_out,
                                 iters_out, st);
  if (e != cudaSuccess) return cuda_fail(e, "svc fit launch");
  return QSVM_OK;
}

int32_t qsvm_svc_decision(const double* Kx, int64_t ldk, int64_t m, const qsvm_svc_problem* problems,
                          int32_t n_problems, const double* b, double* F, void* ws, size_t ws_bytes, void* stream) {
  int32_t rc = svc_check(problems, n_problems);
  if (rc) return rc;
  if (m < 1 || !Kx || !aligned(Kx, 8) || !b || !F || !aligned(F, 8))
    return fail(QSVM_ERR_ARG, "Kx, b and F must be non-null aligned device pointers and m >= 1");
  if (!ws || !aligned(ws, 256) || ws_bytes < svc_table_bytes(n_problems))
    return fail(QSVM_ERR_WORKSPACE, "ws must hold the %zu-byte problem table", svc_table_bytes(n_problems));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  rc = svc_upload(problems, n_problems, ws, false, st);
  if (rc) return rc;
  cudaError_t e = launch_svc_decision(Kx, ldk, m, static_cast<const DevSvcProblem*>(ws), n_problems, b, F, st);
  if (e != cudaSuccess) return cuda_fail(e, "svc decision launch");
  return QSVM_OK;
}

int32_t qsvm_selftest_wait_timeout(int64_t limit_ns, void* stream) {
  if (limit_ns < 1000 || limit_ns > 2000000000LL)
    return fail(QSVM_ERR_ARG, "limit_ns=%lld outside [1e3, 2e9]", (long long)limit_ns);
  cudaError_t e = launch_wait_timeout_selftest((uint64_t)limit_ns, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "self-test launch");
  return QSVM_OK;
}

const char* qsvm_last_error(void) { return g_last_error.c_str(); }

const char* qsvm_version(void) { return "qsvm-gb300 0.1 (sm_103a)"; }

}  // extern "C"

// ---- batch launch for callers that cannot allocate device memory -----------
// Some callers may not allocate device memory at all: real-time or serving
// loops that must not take cudaMalloc's implicit device synchronisation, and
// host programs whose framework allocator already reserves all device memory
// (a second allocator would fail or fragment it).  For them,
// qsvm_kernel_batch_noalloc keeps the batch scratch (job table + work-queue
// head) in a fixed array that lives in this library's device image instead of a
// caller workspace.  The array is loaded with the library on every GPU that uses
// it and stays until the process exits.
namespace {

constexpr int32_t kNoAllocMaxJobs = 1024;
constexpr size_t kNoAllocBytes = 76 * 1024;  // >= the workspace of 1024 jobs
static_assert(ws_total(kNoAllocMaxJobs) <= kNoAllocBytes, "static batch scratch too small for its job limit");

static __device__ __align__(256) uint8_t g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once per
// device (a host-side name of a __device__ array is not a device address).
int32_t noalloc_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return fail(QSVM_ERR_ARG, "device %d beyond the supported %d", dev, kMaxDevices);
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress of the batch scratch");
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return QSVM_OK;
}

}  // namespace

extern "C" int32_t qsvm_kernel_batch_noalloc(const qsvm_job* jobs, int32_t n_jobs, int32_t reps, int32_t precision,
                                             void* stream) {
  if (n_jobs > kNoAllocMaxJobs)
    return fail(QSVM_ERR_WORKSPACE, "n_jobs=%d exceeds the %d jobs the built-in batch scratch holds; use "
                "qsvm_kernel_batch with a workspace", n_jobs, kNoAllocMaxJobs);
  void* ws = nullptr;
  int32_t rc = noalloc_scratch(&ws);
  if (rc) return rc;
  BatchImage img;
  rc = build_batch_image(jobs, n_jobs, reps, precision, ws, kNoAllocBytes, img);
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // the image carries a zero work-queue head, so each call starts its queue at 0
  cudaError_t e = cudaMemcpyAsync(ws, img.bytes.data(), img.bytes.size(), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e, "batch job table upload");
  const BatchArgs a = batch_args(ws, n_jobs, img.total_tiles);
  const PipeCfg pc = current_batch_pipe(reps, precision);
  int grid = 0;
  e = prepare_persistent(1 << reps, precision, pc, img.total_tiles, &grid);
  if (e == cudaSuccess) e = launch_persistent(1 << reps, precision, a, pc, grid, st);
  if (e != cudaSuccess) return cuda_fail(e, "persistent kernel launch");
  return QSVM_OK;
}
