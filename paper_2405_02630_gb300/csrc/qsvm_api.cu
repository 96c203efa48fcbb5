// qsvm_api.cu -- host side of the C ABI declared in include/qsvm.h: argument
// checks, size queries, tile bookkeeping and kernel dispatch.  No allocation.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>

#include "qsvm_common.cuh"

namespace qsvm {
cudaError_t launch_build_mps(const double* X, int64_t N, int n, int reps, int prec, void* mps, cudaStream_t st);
cudaError_t launch_pair(int chi, int prec, const TileArgs& a, int64_t ntiles, cudaStream_t st);
int pair_tile_dim(int chi, int prec);
cudaError_t pair_status(cudaStream_t st, int clear, int32_t* out);
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

// pairs contracted by upper-triangle tile b of a T x T grid over n_points
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
  a.mpsA = a.mpsB = static_cast<const uint8_t*>(mps);
  a.nA = a.nB = n_points;
  a.n = n_qubits;
  a.symmetric = 1;
  a.tile_begin = tile_begin;
  a.tiles_j = T;
  a.K = K;
  a.ldk = ldk;
  a.logK = logK;
  a.ldl = ldl;
  cudaError_t e = launch_pair(chi, precision, a, tile_end - tile_begin, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "pair kernel launch");
  return QSVM_OK;
}

}  // namespace

extern "C" {

size_t qsvm_mps_record_bytes(int32_t reps, int32_t precision) {
  if (reps < 1 || reps > 3 || precision < QSVM_FP64 || precision > QSVM_FP32_SPLIT) return 0;
  return record_bytes(1 << reps, precision);
}

size_t qsvm_mps_bytes(int32_t n_qubits, int32_t reps, int64_t n_points, int32_t precision) {
  if (n_qubits < 1 || n_points < 0) return 0;
  return qsvm_mps_record_bytes(reps, precision) * (size_t)n_qubits * (size_t)n_points;
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
  // boundary r sits at the first tile whose prefix pair count reaches r/world of
  // the total (tiles are whole, so shares differ by at most one tile)
  auto boundary = [&](int64_t r) -> int64_t {
    if (r <= 0) return 0;
    if (r >= world) return total_tiles;
    const double target = (double)total_pairs * (double)r / (double)world;
    int64_t b = 0;
    double acc = 0;
    for (int64_t ti = 0; ti < T; ++ti)
      for (int64_t tj = ti; tj < T; ++tj) {
        if (acc >= target) return b;
        acc += (double)tile_pairs(ti, tj, n_points, tdim);
        ++b;
      }
    return total_tiles;
  };
  *tile_begin = boundary(rank);
  *tile_end = boundary(rank + 1);
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
  a.mpsB = static_cast<const uint8_t*>(mps_b);
  a.nA = n_a;
  a.nB = n_b;
  a.n = n_qubits;
  a.symmetric = 0;
  a.tile_begin = 0;
  a.tiles_j = Tb;
  a.K = K;
  a.ldk = ldk;
  a.logK = logK;
  a.ldl = ldl;
  cudaError_t e = launch_pair(chi, precision, a, Ta * Tb, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "pair kernel launch");
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

const char* qsvm_last_error(void) { return g_last_error.c_str(); }

const char* qsvm_version(void) { return "qsvm-gb300 0.1 (sm_103a)"; }

}  // extern "C"
