// svc.cu -- the support vector classifier trained on a precomputed quantum kernel
// (Sec. 3.2 and Sec. 4.2: the kernel matrix is handed to an SVC; primal Eq. 1-2,
// solved in its dual with the kernel in place of the inner product).
//
// Binary C-SVC dual: minimise 1/2 sum_ij a_i a_j y_i y_j K_ij - sum_i a_i subject to
// 0 <= a_i <= C and sum_i y_i a_i = 0, by sequential minimal optimisation with the
// maximal violating pair: i = argmax_{I_up} -y g, j = argmin_{I_low} -y g, stop when
// the gap m - M falls below tol; the two-variable step is solved exactly and
// clipped to the box.  One CTA solves one binary problem (all of its threads scan
// the candidates and update the gradient), so many problems (one-vs-one classes)
// share a launch; a CTA never waits on another.  K is symmetric, so the gradient
// update reads rows i and j of K contiguously.
#include "qsvm_common.cuh"

namespace qsvm {

struct DevSvcProblem {
  const int64_t* idx;   // n indices into K (training points of this problem)
  const int8_t* y;      // n labels, +1 / -1
  int64_t n;
  double* alpha;        // n outputs
  double* g;            // n doubles of scratch (gradient)
};

namespace {

constexpr int kSvcThreads = 512;

struct ArgBest {
  double v;
  int64_t i;
};

// block-wide argmax (want_max) or argmin, ties to the lower index
__device__ ArgBest block_arg(ArgBest a, bool want_max, ArgBest* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) {
    ArgBest b;
    b.v = __shfl_down_sync(0xffffffffu, a.v, o);
    b.i = __shfl_down_sync(0xffffffffu, a.i, o);
    const bool take = (b.i >= 0) && (a.i < 0 || (want_max ? (b.v > a.v || (b.v == a.v && b.i < a.i))
                                                          : (b.v < a.v || (b.v == a.v && b.i < a.i))));
    if (take) a = b;
  }
  if (lane == 0) sh[warp] = a;
  __syncthreads();
  if (warp == 0) {
    a = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : ArgBest{0.0, -1};
    for (int o = 16; o > 0; o >>= 1) {
      ArgBest b;
      b.v = __shfl_down_sync(0xffffffffu, a.v, o);
      b.i = __shfl_down_sync(0xffffffffu, a.i, o);
      const bool take = (b.i >= 0) && (a.i < 0 || (want_max ? (b.v > a.v || (b.v == a.v && b.i < a.i))
                                                            : (b.v < a.v || (b.v == a.v && b.i < a.i))));
      if (take) a = b;
    }
    if (lane == 0) sh[0] = a;
  }
  __syncthreads();
  const ArgBest r = sh[0];
  __syncthreads();
  return r;
}

__device__ double block_sum(double v, double* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  if (warp == 0) {
    v = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) sh[0] = v;
  }
  __syncthreads();
  const double r = sh[0];
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(kSvcThreads) svc_smo_kernel(const double* __restrict__ K, int64_t ldk,
                                                              const DevSvcProblem* __restrict__ probs, double C,
                                                              double tol, int64_t max_iter, double* b_out,
                                                              int64_t* iters_out) {
  __shared__ ArgBest sh_arg[kSvcThreads / 32];
  __shared__ double sh_sum[kSvcThreads / 32];
  __shared__ double sh_step;
  const DevSvcProblem P = probs[blockIdx.x];
  const int64_t n = P.n;
  for (int64_t t = threadIdx.x; t < n; t += blockDim.x) {
    P.alpha[t] = 0.0;
    P.g[t] = -1.0;
  }
  __syncthreads();
  int64_t it = 0;
  double m = 0.0, M = 0.0;
  for (; it < max_iter; ++it) {
    ArgBest up{-INFINITY, -1}, lo{INFINITY, -1};
    for (int64_t t = threadIdx.x; t < n; t += blockDim.x) {
      const double yt = P.y[t], at = P.alpha[t];
      const double v = -yt * P.g[t];
      const bool in_up = (yt > 0 && at < C) || (yt < 0 && at > 0);
      const bool in_lo = (yt > 0 && at > 0) || (yt < 0 && at < C);
      if (in_up && (up.i < 0 || v > up.v)) up = ArgBest{v, t};
      if (in_lo && (lo.i < 0 || v < lo.v)) lo = ArgBest{v, t};
    }
    const ArgBest bi = block_arg(up, true, sh_arg);
    const ArgBest bj = block_arg(lo, false, sh_arg);
    m = bi.v;
    M = bj.v;
    if (bi.i < 0 || bj.i < 0 || m - M < tol) break;  // uniform across the block
    const int64_t i = bi.i, j = bj.i;
    const int64_t ki = P.idx[i], kj = P.idx[j];
    if (threadIdx.x == 0) {
      double eta = K[ki * ldk + ki] + K[kj * ldk + kj] - 2.0 * K[ki * ldk + kj];
      if (eta <= 1e-12) eta = 1e-12;
      double s = (m - M) / eta;
      const double yi = P.y[i], yj = P.y[j];
      const double si = (yi > 0) ? C - P.alpha[i] : P.alpha[i];
      const double sj = (yj > 0) ? P.alpha[j] : C - P.alpha[j];
      if (s > si) s = si;
      if (s > sj) s = sj;
      P.alpha[i] += yi * s;
      P.alpha[j] -= yj * s;
      sh_step = s;
    }
    __syncthreads();
    const double s = sh_step;
    const double* Ki = K + ki * ldk;
    const double* Kj = K + kj * ldk;
    for (int64_t t = threadIdx.x; t < n; t += blockDim.x) {
      const int64_t kt = P.idx[t];
      P.g[t] += P.y[t] * s * (Ki[kt] - Kj[kt]);
    }
    __syncthreads();
  }
  // bias: mean of -y g over free vectors, else the midpoint of the last bounds
  double sum = 0.0, cnt = 0.0;
  for (int64_t t = threadIdx.x; t < n; t += blockDim.x) {
    const double at = P.alpha[t];
    if (at > 0 && at < C) {
      sum += -P.y[t] * P.g[t];
      cnt += 1.0;
    }
  }
  sum = block_sum(sum, sh_sum);
  cnt = block_sum(cnt, sh_sum);
  if (threadIdx.x == 0) {
    b_out[blockIdx.x] = cnt > 0 ? sum / cnt : 0.5 * (m + M);
    iters_out[blockIdx.x] = it;
  }
}

// F[r * n_probs + p] = sum_i alpha_i y_i Kx[r][idx_i] + b_p
__global__ void svc_decision_kernel(const double* __restrict__ Kx, int64_t ldk, int64_t m,
                                    const DevSvcProblem* __restrict__ probs, int n_probs,
                                    const double* __restrict__ b, double* F) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= m * n_probs) return;
  const int64_t r = g / n_probs;
  const int p = (int)(g - r * n_probs);
  const DevSvcProblem P = probs[p];
  const double* row = Kx + r * ldk;
  double acc = b[p];
  for (int64_t i = 0; i < P.n; ++i) acc = fma(P.alpha[i] * P.y[i], row[P.idx[i]], acc);
  F[g] = acc;
}

}  // namespace

cudaError_t launch_svc_fit(const double* K, int64_t ldk, const DevSvcProblem* probs, int n_probs, double C, double tol,
                           int64_t max_iter, double* b_out, int64_t* iters_out, cudaStream_t st) {
  svc_smo_kernel<<<n_probs, kSvcThreads, 0, st>>>(K, ldk, probs, C, tol, max_iter, b_out, iters_out);
  return cudaGetLastError();
}

cudaError_t launch_svc_decision(const double* Kx, int64_t ldk, int64_t m, const DevSvcProblem* probs, int n_probs,
                                const double* b, double* F, cudaStream_t st) {
  const int64_t total = m * n_probs;
  if (total == 0) return cudaSuccess;
  svc_decision_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(Kx, ldk, m, probs, n_probs, b, F);
  return cudaGetLastError();
}

}  // namespace qsvm
