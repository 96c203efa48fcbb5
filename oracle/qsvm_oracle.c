/*
 * qsvm_oracle.c -- plain, slow, FP64 CPU oracle for quantum-kernel estimation.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this file:
 * only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
 * leg use it.  It shares no code, header, table or helper with the CUDA library.
 *
 * What it computes (arXiv 2405.02630):
 *   K(x_i, x_j) = |<psi(x_j)|psi(x_i)>|^2 = |<0^n| U^dagger(x_j) U(x_i) |0^n>|^2
 *   (Sec. 2, Eq. 3 and Eq. 4), with U(x) the linear-chain feature-map circuit
 *   of Sec. 3.2 (CNOTs in a linear topology, n qubits = n features).  The gate
 *   list per repetition is: H on every qubit, RZ(2 x_k) on every qubit, then for
 *   k = 0..n-2: CNOT(k,k+1) . RZ_{k+1}(2 (pi - x_k)(pi - x_{k+1})) . CNOT(k,k+1).
 *   RZ(theta) = diag(exp(-i theta/2), exp(+i theta/2)).
 *
 * Two independent constructions:
 *   O1  state vector, gate by gate (the recipe of Algorithm 1: build the pair
 *       circuit U^dagger(x_j) U(x_i), simulate it, read the |0..0> amplitude).
 *       Feasible for n <= 20 or so.
 *   O2  closed-form path-sum matrix product state, then the overlap contracted
 *       site by site along the chain (the tensor-network route of Algorithm 2
 *       and Algorithm 3, with the fixed left-to-right order a chain admits).
 *       Any n.  Site tensors are dense [2][chi][chi] with chi = 2^reps, the
 *       environment is rescaled every site by its largest modulus and the
 *       natural log of the scale is accumulated in FP64.
 *
 * Path-sum form used by O2 (derived from the gate list above): with
 * z(b) = 1 - 2b, f_x(s) = sum_k x_k z(s_k) + sum_k (pi-x_k)(pi-x_{k+1}) z(s_k) z(s_{k+1}),
 *   psi_x(s_R) = 2^{-nR/2} sum_{s_1..s_{R-1}} prod_m exp(-i f_x(s_m)) prod_{m>=2} (-1)^{s_{m-1}.s_m}
 * so site k carries the layer spins u = (s_1^k .. s_R^k) on its right bond and
 *   A_k^sigma[t][u] = delta(u_R, sigma) 2^{-R/2} prod_m exp(-i x_k z(u_m))
 *                     * exp(-i (pi-x_{k-1})(pi-x_k) z(t_m) z(u_m))   (k >= 1)
 *                     * prod_{m>=2} (-1)^{u_{m-1} u_m}.
 * Bond index convention here: index = sum_m u_m 2^(m-1) (rep 1 is the low bit).
 *
 * Readings of the paper (it never writes the gate list out):
 *   - K = |amp|^2 per Eq. 3-4 (Algorithms 1-3 store |amp|; sqrt(K) recovers it).
 *   - the diagonal is computed, not set to 1; cross kernels are not symmetrised.
 *
 * flags (bit mask) -- used by the pins:
 *   QO_NO_ENTANGLER  drop the CNOT.RZ.CNOT chain (closed-form product kernels)
 *   QO_PHASE_GATE    use P(2x) = diag(1, e^{2ix}) instead of RZ(2x) (global phase)
 *   QO_MUT_*         test-only planted mistakes; the pins must detect each one
 *
 * Parity status: pinned (see tests/test_oracle_pins.py): O1 vs O2, brute-force
 * Ising sums, closed-form product kernels, K_ii = 1, symmetry, 0 <= K <= 1,
 * positive semidefiniteness, phase-gate invariance, Schmidt-rank bound.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double _Complex cplx;

#define QO_NO_ENTANGLER 1
#define QO_PHASE_GATE 2
#define QO_MUT_ZZ_SIGN 4      /* O1 and O2: wrong sign of the ZZ angle          */
#define QO_MUT_DROP_SIGN 8    /* O2 only: drop the (-1)^{u_{m-1} u_m} factor   */
#define QO_MUT_NO_CONJ 16     /* O2 only: bra site tensor not conjugated        */
#define QO_MUT_SHIFT_COUPLING 32 /* O1 only: couple x_k with x_{k+2}             */

static const double QO_PI = 3.14159265358979323846;

/* ------------------------------------------------------------------ O1 --- */

static void sv_h(cplx* psi, int64_t dim, int q) {
  const double r = 1.0 / sqrt(2.0);
  const int64_t bit = (int64_t)1 << q;
  for (int64_t b = 0; b < dim; ++b) {
    if (b & bit) continue;
    cplx a0 = psi[b], a1 = psi[b | bit];
    psi[b] = r * (a0 + a1);
    psi[b | bit] = r * (a0 - a1);
  }
}

/* diag(exp(-i theta/2), exp(+i theta/2)) on qubit q */
static void sv_rz(cplx* psi, int64_t dim, int q, double theta) {
  const int64_t bit = (int64_t)1 << q;
  const cplx p0 = cexp(-I * theta / 2.0), p1 = cexp(I * theta / 2.0);
  for (int64_t b = 0; b < dim; ++b) psi[b] *= (b & bit) ? p1 : p0;
}

/* diag(1, exp(i lambda)) on qubit q */
static void sv_p(cplx* psi, int64_t dim, int q, double lambda) {
  const int64_t bit = (int64_t)1 << q;
  const cplx p1 = cexp(I * lambda);
  for (int64_t b = 0; b < dim; ++b)
    if (b & bit) psi[b] *= p1;
}

static void sv_cnot(cplx* psi, int64_t dim, int c, int t) {
  const int64_t cb = (int64_t)1 << c, tb = (int64_t)1 << t;
  for (int64_t b = 0; b < dim; ++b) {
    if ((b & cb) && !(b & tb)) {
      cplx tmp = psi[b];
      psi[b] = psi[b | tb];
      psi[b | tb] = tmp;
    }
  }
}

/* one repetition of the feature map, or its inverse (sign = -1 reverses the
 * gate order and negates every angle; H, CNOT are self-inverse). */
static void sv_layer(cplx* psi, int64_t dim, const double* x, int n, int flags, int inverse) {
  const double sgn = inverse ? -1.0 : 1.0;
  const double zz = (flags & QO_MUT_ZZ_SIGN) ? -1.0 : 1.0;
  const int shift = (flags & QO_MUT_SHIFT_COUPLING) ? 2 : 1;
  if (!inverse) {
    for (int q = 0; q < n; ++q) sv_h(psi, dim, q);
    for (int q = 0; q < n; ++q) {
      if (flags & QO_PHASE_GATE) sv_p(psi, dim, q, sgn * 2.0 * x[q]);
      else sv_rz(psi, dim, q, sgn * 2.0 * x[q]);
    }
    if (!(flags & QO_NO_ENTANGLER)) {
      for (int k = 0; k + 1 < n; ++k) {
        int kk = (k + shift < n) ? k + shift : k + 1;
        double phi = zz * 2.0 * (QO_PI - x[k]) * (QO_PI - x[kk]);
        sv_cnot(psi, dim, k, k + 1);
        sv_rz(psi, dim, k + 1, sgn * phi);
        sv_cnot(psi, dim, k, k + 1);
      }
    }
  } else {
    if (!(flags & QO_NO_ENTANGLER)) {
      for (int k = n - 2; k >= 0; --k) {
        int kk = (k + shift < n) ? k + shift : k + 1;
        double phi = zz * 2.0 * (QO_PI - x[k]) * (QO_PI - x[kk]);
        sv_cnot(psi, dim, k, k + 1);
        sv_rz(psi, dim, k + 1, sgn * phi);
        sv_cnot(psi, dim, k, k + 1);
      }
    }
    for (int q = n - 1; q >= 0; --q) {
      if (flags & QO_PHASE_GATE) sv_p(psi, dim, q, sgn * 2.0 * x[q]);
      else sv_rz(psi, dim, q, sgn * 2.0 * x[q]);
    }
    for (int q = n - 1; q >= 0; --q) sv_h(psi, dim, q);
  }
}

/* psi = U(x)|0^n>, psi has 2^n entries (re, im interleaved). Qubit q is bit q. */
int qo_sv_state(const double* x, int n, int reps, int flags, double* psi_out) {
  if (n < 1 || n > 26 || reps < 1) return -1;
  const int64_t dim = (int64_t)1 << n;
  cplx* psi = (cplx*)psi_out;
  memset(psi, 0, sizeof(cplx) * (size_t)dim);
  psi[0] = 1.0;
  for (int r = 0; r < reps; ++r) sv_layer(psi, dim, x, n, flags, 0);
  return 0;
}

/* Algorithm 1 recipe for one pair: simulate U^dagger(x_j) U(x_i)|0^n>, read the
 * all-zero amplitude, K = |amp|^2.  amp_out (nullable) gets (re, im). */
double qo_sv_kernel_pair(const double* xi, const double* xj, int n, int reps, int flags, double* amp_out) {
  if (n < 1 || n > 26 || reps < 1) return -1.0;
  const int64_t dim = (int64_t)1 << n;
  cplx* psi = (cplx*)calloc((size_t)dim, sizeof(cplx));
  if (!psi) return -1.0;
  psi[0] = 1.0;
  for (int r = 0; r < reps; ++r) sv_layer(psi, dim, xi, n, flags, 0);
  for (int r = 0; r < reps; ++r) sv_layer(psi, dim, xj, n, flags, 1);
  cplx amp = psi[0];
  free(psi);
  if (amp_out) {
    amp_out[0] = creal(amp);
    amp_out[1] = cimag(amp);
  }
  return creal(amp) * creal(amp) + cimag(amp) * cimag(amp);
}

/* Gram / cross kernel from per-point state vectors (n small): K[a][b] = |<psi_b|psi_a>|^2 */
int qo_sv_cross(const double* Xa, int64_t na, const double* Xb, int64_t nb, int n, int reps, int flags,
                double* K, int nthreads) {
  if (n < 1 || n > 20 || reps < 1) return -1;
  const int64_t dim = (int64_t)1 << n;
  cplx* Sa = (cplx*)malloc(sizeof(cplx) * (size_t)(dim * na));
  cplx* Sb = (cplx*)malloc(sizeof(cplx) * (size_t)(dim * nb));
  if (!Sa || !Sb) {
    free(Sa);
    free(Sb);
    return -2;
  }
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic)
  for (int64_t a = 0; a < na; ++a) qo_sv_state(Xa + a * n, n, reps, flags, (double*)(Sa + a * dim));
#pragma omp parallel for schedule(dynamic)
  for (int64_t b = 0; b < nb; ++b) qo_sv_state(Xb + b * n, n, reps, flags, (double*)(Sb + b * dim));
#pragma omp parallel for collapse(2) schedule(dynamic)
  for (int64_t a = 0; a < na; ++a)
    for (int64_t b = 0; b < nb; ++b) {
      cplx acc = 0.0;
      const cplx* pa = Sa + a * dim;
      const cplx* pb = Sb + b * dim;
      for (int64_t s = 0; s < dim; ++s) acc += conj(pb[s]) * pa[s];
      K[a * nb + b] = creal(acc) * creal(acc) + cimag(acc) * cimag(acc);
    }
  free(Sa);
  free(Sb);
  return 0;
}

/* ------------------------------------------------------------------ O2 --- */

static int bitm(int idx, int m) { return (idx >> (m - 1)) & 1; } /* layer m = 1..R */

/* Dense closed-form site tensors, A[k][sigma][t][u], chi = 2^reps, padded with
 * zeros: site 0 uses only t = 0 (left bond 1), the last site only u = 0 (right
 * bond 1, layer spins of the last site summed with u_R = sigma). */
int qo_mps_closed_form(const double* x, int n, int reps, int flags, double* A_out) {
  if (n < 1 || reps < 1 || reps > 4) return -1;
  const int R = reps, chi = 1 << reps;
  const size_t site = (size_t)2 * chi * chi;
  cplx* A = (cplx*)A_out;
  memset(A, 0, sizeof(cplx) * site * (size_t)n);
  const double amp0 = pow(2.0, -0.5 * R);
  const double zzs = (flags & QO_MUT_ZZ_SIGN) ? -1.0 : 1.0;
  for (int k = 0; k < n; ++k) {
    const double c = (k > 0 && !(flags & QO_NO_ENTANGLER)) ? zzs * (QO_PI - x[k - 1]) * (QO_PI - x[k]) : 0.0;
    const int tmax = (k > 0) ? chi : 1;
    for (int t = 0; t < tmax; ++t) {
      for (int u = 0; u < chi; ++u) {
        const int sigma = bitm(u, R);
        double ph = 0.0;
        double sign = 1.0;
        for (int m = 1; m <= R; ++m) {
          const double zu = 1.0 - 2.0 * bitm(u, m);
          const double zt = 1.0 - 2.0 * bitm(t, m);
          ph += x[k] * zu + c * zt * zu;
          if (m >= 2 && !(flags & QO_MUT_DROP_SIGN) && bitm(u, m - 1) && bitm(u, m)) sign = -sign;
        }
        const cplx v = sign * amp0 * cexp(-I * ph);
        if (k == n - 1) {
          A[site * k + ((size_t)sigma * chi + t) * chi + 0] += v;
        } else {
          A[site * k + ((size_t)sigma * chi + t) * chi + u] = v;
        }
      }
    }
  }
  return 0;
}

/* Overlap <B|A> of two dense MPS (same n, chi) by site-by-site transfer:
 *   E <- sum_sigma (A^sigma)^T E conj(B^sigma), E_0 = e_0 e_0^T, amp = E_n[0][0].
 * E is divided by its largest modulus after every site and log(scale) summed.
 * Returns K = |amp|^2 (0 on FP64 underflow); logk_out gets ln K (-inf if 0),
 * amp_out (nullable) gets the scaled amplitude and *log_scale_out its log scale. */
double qo_mps_overlap(const double* A_in, const double* B_in, int n, int reps, int flags, double* logk_out,
                      double* amp_out, double* log_scale_out) {
  const int chi = 1 << reps;
  const size_t site = (size_t)2 * chi * chi;
  const cplx* A = (const cplx*)A_in;
  const cplx* B = (const cplx*)B_in;
  cplx E[16 * 16], T[16 * 16], En[16 * 16];
  if (chi > 16) return -1.0;
  memset(E, 0, sizeof(E));
  E[0] = 1.0;
  double L = 0.0;
  for (int k = 0; k < n; ++k) {
    memset(En, 0, sizeof(cplx) * (size_t)chi * chi);
    for (int s = 0; s < 2; ++s) {
      const cplx* As = A + site * k + (size_t)s * chi * chi;
      const cplx* Bs = B + site * k + (size_t)s * chi * chi;
      /* T = (A^s)^T E : T[u][t'] = sum_t A^s[t][u] E[t][t'] */
      for (int u = 0; u < chi; ++u)
        for (int tp = 0; tp < chi; ++tp) {
          cplx acc = 0.0;
          for (int t = 0; t < chi; ++t) acc += As[t * chi + u] * E[t * chi + tp];
          T[u * chi + tp] = acc;
        }
      /* En += T conj(B^s) : En[u][u'] += sum_t' T[u][t'] conj(B^s[t'][u']) */
      for (int u = 0; u < chi; ++u)
        for (int up = 0; up < chi; ++up) {
          cplx acc = 0.0;
          for (int tp = 0; tp < chi; ++tp) {
            cplx b = Bs[tp * chi + up];
            acc += T[u * chi + tp] * ((flags & QO_MUT_NO_CONJ) ? b : conj(b));
          }
          En[u * chi + up] += acc;
        }
    }
    double mx = 0.0;
    for (int e = 0; e < chi * chi; ++e) {
      double a = cabs(En[e]);
      if (a > mx) mx = a;
    }
    if (mx > 0.0) {
      for (int e = 0; e < chi * chi; ++e) E[e] = En[e] / mx;
      L += log(mx);
    } else {
      for (int e = 0; e < chi * chi; ++e) E[e] = 0.0;
    }
  }
  const cplx amp = E[0];
  const double a2 = creal(amp) * creal(amp) + cimag(amp) * cimag(amp);
  const double logk = (a2 > 0.0) ? log(a2) + 2.0 * L : -INFINITY;
  if (logk_out) *logk_out = logk;
  if (amp_out) {
    amp_out[0] = creal(amp);
    amp_out[1] = cimag(amp);
  }
  if (log_scale_out) *log_scale_out = L;
  return (a2 > 0.0) ? exp(logk) : 0.0;
}

/* Kernel matrix over a list of pairs or a full block.
 * K[a*ldk + b] = |<psi(Xb_b)|psi(Xa_a)>|^2 and logK likewise (logK nullable).
 * symmetric != 0 (requires Xa == Xb, na == nb): only a <= b is contracted and
 * the value is mirrored bit-exactly, the diagonal is contracted too. */
int qo_mps_cross(const double* Xa, int64_t na, const double* Xb, int64_t nb, int n, int reps, int flags,
                 int symmetric, double* K, int64_t ldk, double* logK, int64_t ldl, int nthreads) {
  if (n < 1 || reps < 1 || reps > 4) return -1;
  const int chi = 1 << reps;
  const size_t per = (size_t)n * 2 * chi * chi * 2; /* doubles per point */
  double* Ma = (double*)malloc(sizeof(double) * per * (size_t)na);
  double* Mb = symmetric ? Ma : (double*)malloc(sizeof(double) * per * (size_t)nb);
  if (!Ma || !Mb) {
    free(Ma);
    if (!symmetric) free(Mb);
    return -2;
  }
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
#pragma omp parallel for schedule(static)
  for (int64_t a = 0; a < na; ++a) qo_mps_closed_form(Xa + a * n, n, reps, flags, Ma + a * per);
  if (!symmetric) {
#pragma omp parallel for schedule(static)
    for (int64_t b = 0; b < nb; ++b) qo_mps_closed_form(Xb + b * n, n, reps, flags, Mb + b * per);
  }
#pragma omp parallel for collapse(2) schedule(dynamic, 16)
  for (int64_t a = 0; a < na; ++a)
    for (int64_t b = 0; b < nb; ++b) {
      if (symmetric && b < a) continue;
      double lk;
      double k = qo_mps_overlap(Ma + a * per, Mb + b * per, n, reps, flags, &lk, NULL, NULL);
      K[a * ldk + b] = k;
      if (logK) logK[a * ldl + b] = lk;
      if (symmetric && b != a) {
        K[b * ldk + a] = k;
        if (logK) logK[b * ldl + a] = lk;
      }
    }
  free(Ma);
  if (!symmetric) free(Mb);
  return 0;
}

/* Kernel values for an explicit list of pairs (ia[p], ib[p]) into Xa / Xb
 * (the sampled CPU baseline and full-size sampled parity checks). */
int qo_mps_pairs(const double* Xa, const double* Xb, const int64_t* ia, const int64_t* ib, int64_t npairs, int n,
                 int reps, int flags, double* K, double* logK, int nthreads) {
  if (n < 1 || reps < 1 || reps > 4) return -1;
  const int chi = 1 << reps;
  const size_t per = (size_t)n * 2 * chi * chi * 2;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
  int err = 0;
#pragma omp parallel
  {
    double* Ma = (double*)malloc(sizeof(double) * per);
    double* Mb = (double*)malloc(sizeof(double) * per);
    if (!Ma || !Mb) {
#pragma omp atomic write
      err = -2;
    } else {
#pragma omp for schedule(dynamic, 4)
      for (int64_t p = 0; p < npairs; ++p) {
        qo_mps_closed_form(Xa + ia[p] * n, n, reps, flags, Ma);
        qo_mps_closed_form(Xb + ib[p] * n, n, reps, flags, Mb);
        double lk;
        K[p] = qo_mps_overlap(Ma, Mb, n, reps, flags, &lk, NULL, NULL);
        if (logK) logK[p] = lk;
      }
    }
    free(Ma);
    free(Mb);
  }
  return err;
}

int qo_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ----------------------------------------------------------------- SVC --- */
/* Binary C-SVC on a precomputed kernel (the support vector classifier trained on
 * the quantum kernel matrix, Sec. 3.2 / Sec. 4.2; primal of Eq. 1-2 with the
 * kernel in place of the inner product).  Dual: minimise
 *   f(a) = 1/2 sum_ij a_i a_j y_i y_j K_ij - sum_i a_i,  0 <= a_i <= C, sum_i y_i a_i = 0,
 * by sequential minimal optimisation: each step takes the maximal violating pair
 *   i = argmax_{t in I_up} -y_t g_t,  j = argmin_{t in I_low} -y_t g_t
 * (g = gradient, I_up = {a_t < C, y_t = +1} u {a_t > 0, y_t = -1}, I_low the mirror),
 * stops when m(a) - M(a) < tol, and solves the two-variable subproblem exactly
 * with clipping to the box.  K is row-major with leading dimension ldk; idx
 * (nullable) selects the training points of K.  Returns iterations (< 0: error);
 * b is the bias of f(x) = sum_i a_i y_i K(x, x_i) + b. */
long long qo_svc_fit(const double* K, long long ldk, const long long* idx, const signed char* y, long long n,
                     double C, double tol, long long max_iter, double* alpha, double* b_out) {
  double* g = (double*)malloc(sizeof(double) * (size_t)n);
  if (!g) return -2;
  for (long long t = 0; t < n; ++t) {
    alpha[t] = 0.0;
    g[t] = -1.0;
  }
#define KK(a, c) K[(idx ? idx[a] : (a)) * ldk + (idx ? idx[c] : (c))]
  long long it = 0;
  double m = 0.0, M = 0.0;
  for (; it < max_iter; ++it) {
    long long i = -1, j = -1;
    m = -INFINITY;
    M = INFINITY;
    for (long long t = 0; t < n; ++t) {
      const double v = -y[t] * g[t];
      const int up = (y[t] > 0 && alpha[t] < C) || (y[t] < 0 && alpha[t] > 0);
      const int low = (y[t] > 0 && alpha[t] > 0) || (y[t] < 0 && alpha[t] < C);
      if (up && v > m) { m = v; i = t; }
      if (low && v < M) { M = v; j = t; }
    }
    if (i < 0 || j < 0 || m - M < tol) break;
    const double yi = y[i], yj = y[j];
    double eta = KK(i, i) + KK(j, j) - 2.0 * KK(i, j);
    if (eta <= 1e-12) eta = 1e-12;
    /* move along d = (y_i, -y_j) scaled: a_i += y_i s, a_j -= y_j s */
    double s = (m - M) / eta;
    /* box limits for s */
    const double si = (yi > 0) ? C - alpha[i] : alpha[i];
    const double sj = (yj > 0) ? alpha[j] : C - alpha[j];
    if (s > si) s = si;
    if (s > sj) s = sj;
    alpha[i] += yi * s;
    alpha[j] -= yj * s;
    for (long long t = 0; t < n; ++t) g[t] += y[t] * s * (KK(t, i) - KK(t, j));
  }
  /* bias: average of -y_t g_t over free vectors, else midpoint of the bounds */
  double sum = 0.0;
  long long nf = 0;
  for (long long t = 0; t < n; ++t)
    if (alpha[t] > 0 && alpha[t] < C) {
      sum += -y[t] * g[t];
      ++nf;
    }
  *b_out = nf ? sum / (double)nf : 0.5 * (m + M);
#undef KK
  free(g);
  return it;
}

/* f[r] = sum_i alpha_i y_i Kx[r][idx_i] + b for m rows of a cross kernel. */
void qo_svc_decision(const double* Kx, long long ldk, const long long* idx, long long m, const double* alpha,
                     const signed char* y, double b, long long n, double* f) {
  for (long long r = 0; r < m; ++r) {
    double acc = b;
    for (long long i = 0; i < n; ++i) acc += alpha[i] * y[i] * Kx[r * ldk + (idx ? idx[i] : i)];
    f[r] = acc;
  }
}
