// statevector.cu -- GPU state-vector kernel matrix for small n (a validator of the
// MPS path, following the state-vector recipe of Algorithm 1).
//
// Every point's state U(x)|0^n> is simulated gate by gate on its own 2^n complex128
// amplitudes (qubit q is bit q of the basis index): per repetition H on every
// qubit, RZ(2 x_q) on every qubit, then for q = 0..n-2 the literal CNOT(q, q+1),
// RZ_{q+1}(2 (pi - x_q)(pi - x_{q+1})), CNOT(q, q+1).  One launch applies one
// gate to all points.  The Gram K[i][j] = |<psi_j|psi_i>|^2 (Eq. 3-4) is then a
// complex inner product over the 2^n amplitudes, tiled through shared memory in
// FP64.  This shares nothing with the MPS builder or the pair kernels, so the two
// GPU paths check each other.
#include <climits>

#include "qsvm_common.cuh"

namespace qsvm {

namespace {

constexpr int kSvThreads = 256;

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// psi[p] = |0^n>
__global__ void sv_zero_kernel(double2* psi, int64_t total, int64_t dim) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= total) return;
  psi[g] = make_double2((g % dim) == 0 ? 1.0 : 0.0, 0.0);
}

// H on qubit q of every point: butterflies on index pairs (s, s | 2^q), bit q of s = 0.
__global__ void sv_h_kernel(double2* psi, int64_t n_points, int n, int q) {
  const int64_t half = (int64_t)1 << (n - 1);
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n_points * half) return;
  const int64_t p = g / half, k = g - p * half;
  const int64_t lowmask = ((int64_t)1 << q) - 1;
  const int64_t s0 = ((k & ~lowmask) << 1) | (k & lowmask);
  const int64_t s1 = s0 | ((int64_t)1 << q);
  double2* v = psi + (p << n);
  const double2 a = v[s0], b = v[s1];
  const double r = 0.70710678118654752440;
  v[s0] = make_double2((a.x + b.x) * r, (a.y + b.y) * r);
  v[s1] = make_double2((a.x - b.x) * r, (a.y - b.y) * r);
}

// RZ(theta) on qubit q of every point, theta per point:
//   zz == 0: theta = 2 x[p][q];   zz == 1: theta = 2 (pi - x[p][q-1]) (pi - x[p][q]).
// Blocks never straddle points (2^n is a multiple of the block size, or one block per point).
__global__ void sv_rz_kernel(double2* psi, const double* X, int64_t n_points, int n, int q, int zz) {
  const int64_t dim = (int64_t)1 << n;
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t p = ((int64_t)blockIdx.x * blockDim.x) / dim;
  __shared__ double2 ph[2];
  if (threadIdx.x == 0 && p < n_points) {
    const double* x = X + p * n;
    const double theta = zz ? 2.0 * (kPi - x[q - 1]) * (kPi - x[q]) : 2.0 * x[q];
    double s, c;
    sincos(0.5 * theta, &s, &c);
    ph[0] = make_double2(c, -s);  // e^{-i theta/2} on bit 0
    ph[1] = make_double2(c, s);   // e^{+i theta/2} on bit 1
  }
  __syncthreads();
  if (g >= n_points * dim) return;
  const int64_t s = g - p * dim;
  psi[g] = cmul(psi[g], ph[(s >> q) & 1]);
}

// CNOT(c, t) on every point: swap amplitudes s and s ^ 2^t where bit c of s is 1 and bit t is 0.
__global__ void sv_cnot_kernel(double2* psi, int64_t n_points, int n, int c, int t) {
  const int64_t dim = (int64_t)1 << n;
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n_points * dim) return;
  const int64_t s = g & (dim - 1);
  if (((s >> c) & 1) && !((s >> t) & 1)) {
    const int64_t g2 = g | ((int64_t)1 << t);
    const double2 a = psi[g], b = psi[g2];
    psi[g] = b;
    psi[g2] = a;
  }
}

// K[i][j] = |sum_s conj(psi_j[s]) psi_i[s]|^2 for one 16 x 16 tile (symmetric: tiles
// ti <= tj, mirrored; the mirror is the same double).  Amplitudes are staged 32 at a
// time for the tile's 32 points.
constexpr int kSvTile = 16, kSvChunk = 32;
__global__ void __launch_bounds__(kSvTile * kSvTile) sv_gram_kernel(const double2* __restrict__ psi, int64_t n_points,
                                                                    int n, int64_t T, double* K, int64_t ldk) {
  __shared__ double2 sa[kSvTile][kSvChunk + 1], sb[kSvTile][kSvChunk + 1];
  int64_t ti, tj;
  sym_tile_decode(blockIdx.x, T, ti, tj);
  const int64_t dim = (int64_t)1 << n;
  const int tx = threadIdx.x % kSvTile, ty = threadIdx.x / kSvTile;
  const int64_t i = ti * kSvTile + ty, j = tj * kSvTile + tx;
  double re = 0.0, im = 0.0;
  for (int64_t s0 = 0; s0 < dim; s0 += kSvChunk) {
    // 256 threads load 16 points x 32 amplitudes for each side
    for (int e = threadIdx.x; e < kSvTile * kSvChunk; e += blockDim.x) {
      const int pt = e / kSvChunk, k = e % kSvChunk;
      const int64_t pa = ti * kSvTile + pt, pb = tj * kSvTile + pt, s = s0 + k;
      sa[pt][k] = (pa < n_points && s < dim) ? psi[(pa << n) + s] : make_double2(0.0, 0.0);
      sb[pt][k] = (pb < n_points && s < dim) ? psi[(pb << n) + s] : make_double2(0.0, 0.0);
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < kSvChunk; ++k) {
      const double2 a = sa[ty][k], b = sb[tx][k];  // conj(b) a
      re = fma(b.x, a.x, re);
      re = fma(b.y, a.y, re);
      im = fma(b.x, a.y, im);
      im = fma(-b.y, a.x, im);
    }
    __syncthreads();
  }
  if (i < n_points && j < n_points && (ti != tj || ty <= tx)) {
    const double k2 = re * re + im * im;
    K[i * ldk + j] = k2;
    K[j * ldk + i] = k2;
  }
}

unsigned blocks_for(int64_t work) { return (unsigned)((work + kSvThreads - 1) / kSvThreads); }

}  // namespace

// Simulates every point's circuit into psi (n_points x 2^n complex128) and writes the Gram.
cudaError_t launch_sv_gram(const double* X, int64_t N, int n, int reps, void* ws, double* K, int64_t ldk,
                           cudaStream_t st) {
  double2* psi = static_cast<double2*>(ws);
  const int64_t dim = (int64_t)1 << n;
  const int64_t total = N * dim;
  // the diagonal-gate kernel reads the point of a block from its first thread: a
  // block must not straddle two points, so 2^n >= block size or one block per point
  const int rz_threads = dim >= kSvThreads ? kSvThreads : (int)dim;
  const unsigned rz_blocks = (unsigned)((total + rz_threads - 1) / rz_threads);
  sv_zero_kernel<<<blocks_for(total), kSvThreads, 0, st>>>(psi, total, dim);
  for (int r = 0; r < reps; ++r) {
    for (int q = 0; q < n; ++q) sv_h_kernel<<<blocks_for(N * (dim / 2)), kSvThreads, 0, st>>>(psi, N, n, q);
    for (int q = 0; q < n; ++q) sv_rz_kernel<<<rz_blocks, rz_threads, 0, st>>>(psi, X, N, n, q, 0);
    for (int q = 0; q + 1 < n; ++q) {
      sv_cnot_kernel<<<blocks_for(total), kSvThreads, 0, st>>>(psi, N, n, q, q + 1);
      sv_rz_kernel<<<rz_blocks, rz_threads, 0, st>>>(psi, X, N, n, q + 1, 1);
      sv_cnot_kernel<<<blocks_for(total), kSvThreads, 0, st>>>(psi, N, n, q, q + 1);
    }
  }
  const int64_t T = (N + kSvTile - 1) / kSvTile;
  const int64_t tiles = T * (T + 1) / 2;
  if (tiles > INT_MAX) return cudaErrorInvalidValue;
  sv_gram_kernel<<<(unsigned)tiles, kSvTile * kSvTile, 0, st>>>(psi, N, n, T, K, ldk);
  return cudaGetLastError();
}

}  // namespace qsvm
