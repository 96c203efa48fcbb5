// build_mps.cu -- K1: exact MPS of U(x)|0^n> for every data point, in FP64.
//
// The circuit is the linear-chain feature map of arXiv 2405.02630 Sec. 3.2 (one
// qubit per feature, CNOTs in a linear topology); per repetition: H on every
// qubit, RZ(2 x_k) on every qubit, then CNOT(k,k+1) . RZ_{k+1}(2 theta_k) .
// CNOT(k,k+1) for k = 0..n-2 with theta_k = (pi - x_k)(pi - x_{k+1}).
//
// Every gate acts on at most the bond next to a site, so each site tensor can be
// built on its own from (x_{k-1}, x_k): the builder starts each site in |0>
// with bond dimension 1 and applies, per repetition,
//   H        on the physical index;
//   RZ(2x_k) on the physical index: diag(e^{-i x_k}, e^{+i x_k});
//   the CNOT.RZ.CNOT chain of that repetition as one bond-2 diagonal MPO.  The
//   block on (k-1, k) equals exp(-i theta_{k-1} Z_{k-1} Z_k); as an MPO the left
//   site copies its spin onto the shared bond (right bond grows by a bit b equal
//   to the spin) and the right site multiplies by exp(-i theta z(a) z(sigma))
//   where a is that copied spin (left bond grows by the bit a).
// After reps repetitions both bonds have dimension 2^reps (site 0: left bond 1;
// last site: right bond 1), with rep 1 in the most significant bit.  The last
// repetition's copied bit is the low bit of the right bond and equals the
// physical index, which is what the block layout of the record relies on.
//
// The low bit c of the left bond (the left neighbour's last-repetition spin)
// enters the site tensor only through the last repetition's ZZ phase
// exp(-i theta z(c) z(sigma)), so the rows with c = 1 are the rows with c = 0
// times exp(2 i theta z(sigma)).  The record therefore keeps the c = 0 blocks
// a_0s and the phase r = exp(2 i theta_{k-1}) (1 at site 0, where only t = 0
// exists); the contraction applies the c = 1 half through r.
#include "qsvm_common.cuh"

namespace qsvm {

struct cd {
  double re, im;
};
__device__ __forceinline__ cd cmul(cd a, cd b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }

// Store one complex value at byte offset off of a record, in the requested
// format: FP64 once as (re, im); FP32 formats in both forms (recA: a-form
// (A, iA); recB: b-form (conj A, i conj A)), the split format as hi then lo parts.
__device__ __forceinline__ void store_forms(uint8_t* pa, uint8_t* pb, float re, float im) {
  reinterpret_cast<float4*>(pa)[0] = make_float4(re, im, -im, re);
  reinterpret_cast<float4*>(pb)[0] = make_float4(re, -im, im, re);
}

template <int CHI, int PREC>
__device__ __forceinline__ void store_entry(uint8_t* recA, uint8_t* recB, int off, cd v) {
  using Rec = Record<CHI, PREC>;
  if constexpr (PREC == QSVM_FP64) {
    reinterpret_cast<double2*>(recA + off)[0] = make_double2(v.re, v.im);
  } else if constexpr (PREC == QSVM_FP32) {
    store_forms(recA + off, recB + off, __double2float_rn(v.re), __double2float_rn(v.im));
  } else {
    // hi: nearest multiple of 2^-kGridT (exact in double and in float since
    // |v| <= 1); lo: the remainder rounded to float.  Block entries keep their
    // lo part kPartBytes after the hi part; the phase keeps it in the next entry.
    constexpr double s = (double)(1 << kGridT);
    const double hr = rint(v.re * s) / s, hi = rint(v.im * s) / s;
    const int lo_off = off < Rec::kPhaseOff ? Rec::kPartBytes : Rec::kEntryBytes;
    store_forms(recA + off, recB + off, (float)hr, (float)hi);
    store_forms(recA + off + lo_off, recB + off + lo_off, __double2float_rn(v.re - hr), __double2float_rn(v.im - hi));
  }
}

// Row t of the site tensor: v[sigma][u] after all repetitions.
// LAST: the site has no right neighbour (no copy onto a right bond).
template <int R, bool LAST>
__device__ __forceinline__ void site_row(int t, bool has_left, cd rz0, cd zzp, cd zzm, cd (&v)[2][1 << R]) {
  constexpr int CHI = 1 << R;
  const double r2 = 0.70710678118654752440;
#pragma unroll
  for (int r = 0; r < CHI; ++r) v[0][r] = v[1][r] = cd{0.0, 0.0};
  v[0][0] = cd{1.0, 0.0};
#pragma unroll
  for (int m = 1; m <= R; ++m) {
    const int d = LAST ? 1 : (1 << (m - 1));  // right-bond dimension before this rep
    // H on the physical index
#pragma unroll
    for (int r = 0; r < d; ++r) {
      const cd a = v[0][r], b = v[1][r];
      v[0][r] = cd{(a.re + b.re) * r2, (a.im + b.im) * r2};
      v[1][r] = cd{(a.re - b.re) * r2, (a.im - b.im) * r2};
    }
    // RZ(2 x_k): sigma = 0 gets e^{-i x}, sigma = 1 gets e^{+i x}
    const cd rz1 = cd{rz0.re, -rz0.im};
#pragma unroll
    for (int r = 0; r < d; ++r) {
      v[0][r] = cmul(v[0][r], rz0);
      v[1][r] = cmul(v[1][r], rz1);
    }
    // ZZ block with the left neighbour: exp(-i theta z(a) z(sigma)), a = bit of t
    if (has_left) {
      const int a = (t >> (R - m)) & 1;
      const cd p0 = a ? zzm : zzp;             // sigma = 0: exp(-i theta z(a))
      const cd p1 = cd{p0.re, -p0.im};         // sigma = 1: exp(+i theta z(a))
#pragma unroll
      for (int r = 0; r < d; ++r) {
        v[0][r] = cmul(v[0][r], p0);
        v[1][r] = cmul(v[1][r], p1);
      }
    }
    // copy the spin onto the right bond: v'[sigma][2r + sigma] = v[sigma][r]
    if (!LAST) {
#pragma unroll
      for (int r = d - 1; r >= 0; --r) {
        const cd a = v[0][r], b = v[1][r];
        v[0][2 * r] = a;
        v[0][2 * r + 1] = cd{0.0, 0.0};
        v[1][2 * r] = cd{0.0, 0.0};
        v[1][2 * r + 1] = b;
      }
    }
  }
}

// Phase-form records (reps = 2, plain FP32).
// At reps = 2, multiplying out the gates of one site gives
// A^s[2q+c][2p+s] = (1/2) (-1)^{p s} e^{-i x (z(p) + z(s))} e^{-i theta (z(q) z(p) + z(c) z(s))}
// (z(b) = 1 - 2b; the two RZ layers, the two ZZ layers with the left neighbour's
// layer spins q, c, and the Hadamard sign between the layers), so with
// P = e^{-i x_k}, T = e^{-i theta_{k-1}} every entry is +-1/2 times one of 1,
// T^2, P^2, P^2 T^2 or a conjugate: the record keeps those three phases, read off
// the entries the gate-by-gate build produces.  The last site keeps the same
// tensor with its right bond open (the contraction sums it at the end).  FP64 and
// split FP32 store the gauged form made from the same phases (qsvm_common.cuh).
__device__ __forceinline__ void store_phase(uint8_t* rec, int v, cd z) {  // reps = 2, plain FP32
  using Rec = Record<4, QSVM_FP32>;
  store_forms(rec + Rec::off(v, 0), rec + Rec::off(v, 1), __double2float_rn(z.re), __double2float_rn(z.im));
}

// Gauged-form record (split FP32, reps = 2 and 3) of site k of point i: alpha and beta,
// hi on 2^-kGridT and the lo remainder, a-form entries into the row-side array and
// b-form entries into the column-side array (n + 1 records per point each).
// The same values in FP64: (re, im) doubles of alpha and beta, one array.
__device__ __forceinline__ void store_gauged_fp64(uint8_t* mps, int n, int64_t i, int k, cd alpha, cd beta) {
  using Rec = Record<4, QSVM_FP64>;
  double2* rec = reinterpret_cast<double2*>(mps + (i * record_sites(n, 4, QSVM_FP64) + k) * Rec::kBytes);
  rec[0] = make_double2(alpha.re, alpha.im);
  rec[1] = make_double2(beta.re, beta.im);
}

__device__ __forceinline__ void store_gauged(uint8_t* mps, int64_t n_points, int n, int64_t i, int k, cd alpha,
                                             cd beta) {
  using Rec = Record<4, QSVM_FP32_SPLIT>;
  const int64_t sites = record_sites(n, 4, QSVM_FP32_SPLIT);
  uint8_t* pa = mps + (i * sites + k) * Rec::kBytes;
  uint8_t* pb = pa + n_points * sites * Rec::kBytes;
  constexpr double sc = (double)(1 << kGridT);
  const cd z[2] = {alpha, beta};
#pragma unroll
  for (int v = 0; v < 2; ++v) {
    const double hr = rint(z[v].re * sc) / sc, hi = rint(z[v].im * sc) / sc;
    store_forms(pa + Rec::off(v, 0), pb + Rec::off(v, 0), (float)hr, (float)hi);
    store_forms(pa + Rec::off(v, 1), pb + Rec::off(v, 1), __double2float_rn(z[v].re - hr),
                __double2float_rn(z[v].im - hi));
  }
}

// The gate parameters of site k of point i: rz0 = e^{-i x_k}; zzp, zzm = exp(-+i theta_{k-1}).
__device__ __forceinline__ void site_params(const double* X, int64_t i, int n, int k, cd& rz0, cd& zzp, cd& zzm) {
  const double xk = X[i * n + k];
  double sx, cx;
  sincos(xk, &sx, &cx);
  rz0 = cd{cx, -sx};
  zzp = zzm = cd{1.0, 0.0};
  if (k > 0) {
    const double th = (kPi - X[i * n + k - 1]) * (kPi - xk);
    double st, ct;
    sincos(th, &st, &ct);
    zzp = cd{ct, -st};  // a = 0: z(a) = +1 -> exp(-i theta) for sigma = 0
    zzm = cd{ct, st};   // a = 1: z(a) = -1 -> exp(+i theta) for sigma = 0
  }
}

// The three phases V0 = T^2, V1 = P^2, V2 = P^2 T^2 of site k (reps = 2), read off
// rows t = 0 and t = 2 of the gate-by-gate build (right bond open, also at the last
// site): a_00[0][0] = V2 / 2, a_00[1][0] = V1 / 2, a_00[1][1] = V0 / 2.  Site 0 has
// only t = 0; there T = 1, so V0 = 1 and V1 = V2.
__device__ __forceinline__ void phases_r2(const double* X, int64_t i, int n, int k, cd& V0, cd& V1, cd& V2) {
  cd rz0, zzp, zzm;
  site_params(X, i, n, k, rz0, zzp, zzm);
  cd v[2][4];
  site_row<2, false>(0, k > 0, rz0, zzp, zzm, v);
  V2 = cd{2.0 * v[0][0].re, 2.0 * v[0][0].im};
  V1 = V2;
  V0 = cd{1.0, 0.0};
  if (k > 0) {
    site_row<2, false>(2, true, rz0, zzp, zzm, v);
    V1 = cd{2.0 * v[0][0].re, 2.0 * v[0][0].im};
    V0 = cd{2.0 * v[0][2].re, 2.0 * v[0][2].im};
  }
}

__device__ __forceinline__ cd conj_(cd a) { return cd{a.re, -a.im}; }

template <int R, int PREC>
__global__ void __launch_bounds__(256) build_mps_kernel(const double* __restrict__ X, int64_t n_points, int n,
                                                        uint8_t* __restrict__ mps) {
  constexpr int CHI = 1 << R;
  using Rec = Record<CHI, PREC>;
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= n_points * (int64_t)n) return;
  const int64_t i = gid / n;
  const int k = (int)(gid - i * n);
  cd rz0, zzp, zzm;
  site_params(X, i, n, k, rz0, zzp, zzm);
  const bool has_left = k > 0;
  if constexpr (R >= 2 && PREC != QSVM_FP32) {
    // gauged form (FP64 and split FP32 at reps = 2 and 3): alpha_k = conj(V2^{k-1} V0^k),
    // beta_k = conj(V2^{k-1}) V0^k with the reps = 2 phases (V2^{-1} = 1); the thread of
    // the last site also writes the virtual site n
    cd V0, V1, V2, P0, P1, V2p = cd{1.0, 0.0};
    phases_r2(X, i, n, k, V0, V1, V2);
    if (has_left) phases_r2(X, i, n, k - 1, P0, P1, V2p);
    const cd c = conj_(V2p);
    if constexpr (PREC == QSVM_FP64) {
      store_gauged_fp64(mps, n, i, k, cmul(c, conj_(V0)), cmul(c, V0));
      if (k == n - 1) store_gauged_fp64(mps, n, i, n, conj_(V2), conj_(V2));
    } else {
      store_gauged(mps, n_points, n, i, k, cmul(c, conj_(V0)), cmul(c, V0));
      if (k == n - 1) store_gauged(mps, n_points, n, i, n, conj_(V2), conj_(V2));
    }
  } else if constexpr (R == 2) {
    cd V0, V1, V2;
    phases_r2(X, i, n, k, V0, V1, V2);
    uint8_t* rec = mps + gid * Record<4, PREC>::kBytes;
    store_phase(rec, 0, V0);
    store_phase(rec, 1, V1);
    store_phase(rec, 2, V2);
  } else {
    uint8_t* recA = mps + gid * Rec::kBytes;
    uint8_t* recB = recA + (Rec::kForms == 2 ? n_points * (int64_t)n * Rec::kBytes : 0);
    const bool last = (k == n - 1);
    constexpr int H = CHI / 2;
    // rows t = 2q (c = 0) of both blocks s
    for (int q = 0; q < H; ++q) {
      const int t = 2 * q;
      cd v[2][CHI];
      if (!has_left && t > 0) {
#pragma unroll
        for (int u = 0; u < CHI; ++u) v[0][u] = v[1][u] = cd{0.0, 0.0};
      } else if (last) {
        site_row<R, true>(t, has_left, rz0, zzp, zzm, v);
      } else {
        site_row<R, false>(t, has_left, rz0, zzp, zzm, v);
      }
#pragma unroll
      for (int u = 0; u < CHI; ++u) {
        const int s = u & 1, p = u >> 1;
        cd val;
        if (last) val = (u < 2) ? v[u][0] : cd{0.0, 0.0};
        else val = v[s][u];
        store_entry<CHI, PREC>(recA, recB, s * Rec::kBlockStride + (q * H + p) * Rec::kEntryBytes, val);
      }
    }
    // r = exp(2 i theta) = (zzm)^2: the ratio of the c = 1 rows to the c = 0 rows for sigma = 0
    store_entry<CHI, PREC>(recA, recB, Rec::kPhaseOff, cmul(zzm, zzm));
  }
}

template <int R, int PREC>
static cudaError_t launch_build_t(const double* X, int64_t N, int n, void* mps, cudaStream_t st) {
  const int64_t total = N * (int64_t)n;
  const int threads = 256;
  const int64_t blocks = (total + threads - 1) / threads;
  build_mps_kernel<R, PREC><<<(unsigned)blocks, threads, 0, st>>>(X, N, n, static_cast<uint8_t*>(mps));
  return cudaGetLastError();
}

template <int R>
static cudaError_t launch_build_r(const double* X, int64_t N, int n, int prec, void* mps, cudaStream_t st) {
  switch (prec) {
    case QSVM_FP64: return launch_build_t<R, QSVM_FP64>(X, N, n, mps, st);
    case QSVM_FP32: return launch_build_t<R, QSVM_FP32>(X, N, n, mps, st);
    default: return launch_build_t<R, QSVM_FP32_SPLIT>(X, N, n, mps, st);
  }
}

cudaError_t launch_build_mps(const double* X, int64_t N, int n, int reps, int prec, void* mps, cudaStream_t st) {
  switch (reps) {
    case 1: return launch_build_r<1>(X, N, n, prec, mps, st);
    case 2: return launch_build_r<2>(X, N, n, prec, mps, st);
    default: return launch_build_r<3>(X, N, n, prec, mps, st);
  }
}

}  // namespace qsvm
