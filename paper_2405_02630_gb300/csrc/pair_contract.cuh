// pair_contract.cuh -- all-pairs transfer-matrix contraction (K3, FP32, split FP32).
//
// For a pair (i, j) the overlap <psi_j|psi_i> of arXiv 2405.02630 Eq. 4 is
// contracted along the chain (the tensor-network kernel of Algorithm 2, whose
// path is the fixed left-to-right order on a chain):
//     E_0 = e_0 e_0^T,   E_{k+1} = sum_sigma (A_{i,k}^sigma)^T E_k conj(A_{j,k}^sigma),
//     amp = trace(E_n)   (the last site's right bond carries sigma).
// The feature map ends on a diagonal layer, so A^sigma[t][u] vanishes unless the
// low bit of u equals sigma; E is then block diagonal in (t & 1, t' & 1) and the
// update splits into four chi/2-sized products per site (block b = 2c + s):
//     E'_s = sum_c a_cs^T E_c conj(b_cs)            (chi^3 complex MACs per site)
// which is a quarter of the dense 4 chi^3.
//
// One CTA owns a TI x TI tile of pairs, one thread per pair, E in registers for
// all n sites.  The tile's 2*TI points stream their site records through shared
// memory in chunks of S sites: one thread issues one bulk (TMA) copy per point
// and chunk, completion is tracked by an mbarrier per stage, two stages in flight.
//
// Renormalisation: E is scaled by an exact power of two 2^-e (max |component| of
// E into [0.5, 1)) and e is accumulated in an integer, so the scale is exact.
#pragma once

#include <math.h>

#include "qsvm_common.cuh"

namespace qsvm {

// ---------------------------------------------------------- loads ---------
template <int H>
__device__ __forceinline__ void load_block_f(const uint8_t* p, float2 (&d)[H][H]) {
  if constexpr ((H * H) % 2 == 0) {
    const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
    for (int e = 0; e < H * H / 2; ++e) {
      const float4 v = q[e];
      d[(2 * e) / H][(2 * e) % H] = make_float2(v.x, v.y);
      d[(2 * e + 1) / H][(2 * e + 1) % H] = make_float2(v.z, v.w);
    }
  } else {
    const float2* q = reinterpret_cast<const float2*>(p);
#pragma unroll
    for (int e = 0; e < H * H; ++e) d[e / H][e % H] = q[e];
  }
}

template <int H>
__device__ __forceinline__ void load_block_d(const uint8_t* p, double2 (&d)[H][H]) {
  const double2* q = reinterpret_cast<const double2*>(p);
#pragma unroll
  for (int e = 0; e < H * H; ++e) d[e / H][e % H] = q[e];
}

// --------------------------------------------------------- engines --------
template <int CHI, int PREC>
struct Engine;

// FP64 everywhere (the parity path).
template <int CHI>
struct Engine<CHI, QSVM_FP64> {
  static constexpr int H = CHI / 2;
  static constexpr int kRenormEvery = 8;
  using Rec = Record<CHI, QSVM_FP64>;
  double2 E[2][H][H];
  int L;

  __device__ __forceinline__ void init() {
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int q = 0; q < H; ++q)
#pragma unroll
        for (int r = 0; r < H; ++r) E[c][q][r] = make_double2(0.0, 0.0);
    E[0][0][0].x = 1.0;
    L = 0;
  }

  __device__ __forceinline__ void site(const uint8_t* ra, const uint8_t* rb) {
    double2 N[2][H][H];
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int p = 0; p < H; ++p)
#pragma unroll
        for (int r = 0; r < H; ++r) N[s][p][r] = make_double2(0.0, 0.0);
#pragma unroll
    for (int s = 0; s < 2; ++s) {
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        double2 a[H][H], b[H][H];
        load_block_d<H>(ra + (2 * c + s) * Rec::kBlockBytes, a);
        load_block_d<H>(rb + (2 * c + s) * Rec::kBlockBytes, b);
#pragma unroll
        for (int p = 0; p < H; ++p) {
          double2 X[H];
#pragma unroll
          for (int r = 0; r < H; ++r) {  // X[r] = sum_q a[q][p] E_c[q][r]
            double xr = 0.0, xi = 0.0;
#pragma unroll
            for (int q = 0; q < H; ++q) {
              const double2 A = a[q][p], e = E[c][q][r];
              xr = fma(A.x, e.x, xr);
              xr = fma(-A.y, e.y, xr);
              xi = fma(A.x, e.y, xi);
              xi = fma(A.y, e.x, xi);
            }
            X[r] = make_double2(xr, xi);
          }
#pragma unroll
          for (int pp = 0; pp < H; ++pp) {  // N_s[p][pp] += sum_r X[r] conj(b[r][pp])
            double nr = N[s][p][pp].x, ni = N[s][p][pp].y;
#pragma unroll
            for (int r = 0; r < H; ++r) {
              const double2 B = b[r][pp];
              nr = fma(X[r].x, B.x, nr);
              nr = fma(X[r].y, B.y, nr);
              ni = fma(X[r].y, B.x, ni);
              ni = fma(-X[r].x, B.y, ni);
            }
            N[s][p][pp] = make_double2(nr, ni);
          }
        }
      }
    }
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int p = 0; p < H; ++p)
#pragma unroll
        for (int r = 0; r < H; ++r) E[s][p][r] = N[s][p][r];
  }

  __device__ __forceinline__ void renorm() {
    double m = 0.0;
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int p = 0; p < H; ++p)
#pragma unroll
        for (int r = 0; r < H; ++r) m = fmax(m, fmax(fabs(E[s][p][r].x), fabs(E[s][p][r].y)));
    if (!(m > 0.0) || !isfinite(m)) return;
    int e;
    frexp(m, &e);
    if (e < -1000) e = -1000;
    const double sc = ldexp(1.0, -e);
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int p = 0; p < H; ++p)
#pragma unroll
        for (int r = 0; r < H; ++r) {
          E[s][p][r].x *= sc;
          E[s][p][r].y *= sc;
        }
    L += e;
  }

  __device__ __forceinline__ void amplitude(double& re, double& im) const {
    re = E[0][0][0].x + E[1][0][0].x;
    im = E[0][0][0].y + E[1][0][0].y;
  }
};

// Plain FP32: same algebra in float, renormalised every 4 sites.
template <int CHI>
struct Engine<CHI, QSVM_FP32> {
  static constexpr int H = CHI / 2;
  static constexpr int kRenormEvery = 4;
  using Rec = Record<CHI, QSVM_FP32>;
  float2 E[2][H][H];
  int L;

  __device__ __forceinline__ void init() {
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int q = 0; q < H; ++q)
#pragma unroll
        for (int r = 0; r < H; ++r) E[c][q][r] = make_float2(0.f, 0.f);
    E[0][0][0].x = 1.f;
    L = 0;
  }

  __device__ __forceinline__ void site(const uint8_t* ra, const uint8_t* rb) {
    float2 N[2][H][H];
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int p = 0; p < H; ++p)
#pragma unroll
        for (int r = 0; r < H; ++r) N[s][p][r] = make_float2(0.f, 0.f);
#pragma unroll
    for (int s = 0; s < 2; ++s) {
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        float2 a[H][H], b[H][H];
        load_block_f<H>(ra + (2 * c + s) * Rec::kBlockBytes, a);
        load_block_f<H>(rb + (2 * c + s) * Rec::kBlockBytes, b);
#pragma unroll
        for (int p = 0; p < H; ++p) {
          float2 X[H];
#pragma unroll
          for (int r = 0; r < H; ++r) {
            float xr = 0.f, xi = 0.f;
#pragma unroll
            for (int q = 0; q < H; ++q) {
              const float2 A = a[q][p], e = E[c][q][r];
              xr = fmaf(A.x, e.x, xr);
              xr = fmaf(-A.y, e.y, xr);
              xi = fmaf(A.x, e.y, xi);
              xi = fmaf(A.y, e.x, xi);
            }
            X[r] = make_float2(xr, xi);
          }
#pragma unroll
          for (int pp = 0; pp < H; ++pp) {
            float nr = N[s][p][pp].x, ni = N[s][p][pp].y;
#pragma unroll
            for (int r = 0; r < H; ++r) {
              const float2 B = b[r][pp];
              nr = fmaf(X[r].x, B.x, nr);
              nr = fmaf(X[r].y, B.y, nr);
              ni = fmaf(X[r].y, B.x, ni);
              ni = fmaf(-X[r].x, B.y, ni);
            }
            N[s][p][pp] = make_float2(nr, ni);
          }
        }
      }
    }
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int p = 0; p < H; ++p)
#pragma unroll
        for (int r = 0; r < H; ++r) E[s][p][r] = N[s][p][r];
  }

  __device__ __forceinline__ void renorm() {
    float m = 0.f;
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int p = 0; p < H; ++p)
#pragma unroll
        for (int r = 0; r < H; ++r) m = fmaxf(m, fmaxf(fabsf(E[s][p][r].x), fabsf(E[s][p][r].y)));
    if (!(m > 0.f) || !isfinite(m)) return;
    int e;
    frexpf(m, &e);
    float sc;
    if (e < -120) {  // subnormal territory: scale in two exact steps
#pragma unroll
      for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int p = 0; p < H; ++p)
#pragma unroll
          for (int r = 0; r < H; ++r) {
            E[s][p][r].x *= pow2f(100);
            E[s][p][r].y *= pow2f(100);
          }
      L -= 100;
      e += 100;
    }
    sc = pow2f(-e);
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int p = 0; p < H; ++p)
#pragma unroll
        for (int r = 0; r < H; ++r) {
          E[s][p][r].x *= sc;
          E[s][p][r].y *= sc;
        }
    L += e;
  }

  __device__ __forceinline__ void amplitude(double& re, double& im) const {
    re = (double)E[0][0][0].x + (double)E[1][0][0].x;
    im = (double)E[0][0][0].y + (double)E[1][0][0].y;
  }
};

// Split FP32.  Every value v is carried as hi + lo: hi on a fixed binary grid,
// lo the FP32 remainder.  Products of hi parts and their short sums are exact
// in FP32 FMAs because they stay on a common grid below 2^24 units:
//   step 1  X = a^T E_c:   hi(a) on 2^-11 with |hi(a)| <= 2^{-reps/2} + 2^-12,
//           hi(E) on 2^-10 with |hi(E)| <= 1 + 2^-11 (E renormalised every site),
//           2*(chi/2) real products per sum  ->  < 6.0e6 units of 2^-21 (chi <= 8);
//   step 2  E' = sum_c X conj(b):  hi(X) on 2^-GX (GX = 9, or 8 for chi = 8) with
//           |X| <= chi * 2^{-reps/2} (<= 2.83), hi(b) on 2^-11, 4*(chi/2) real
//           products  ->  < 8.4e6 units of 2^-(GX+11)  (2^24 = 1.68e7).
// The lo terms (hi(a) lo(E) + lo(a) full(E), and the same for step 2) are
// about 2^-11 of the result, so their FP32 rounding costs ~2^-35 relative per
// site; nothing else is rounded.  This is the split hi+lo compensated product
// carried out on the FP32 pipe.
template <int CHI>
struct Engine<CHI, QSVM_FP32_SPLIT> {
  static constexpr int H = CHI / 2;
  static constexpr int GX = grid_x(CHI);
  static constexpr int kRenormEvery = 1;  // built into site()
  using Rec = Record<CHI, QSVM_FP32_SPLIT>;
  float2 Eh[2][H][H], El[2][H][H];
  int L;

  __device__ __forceinline__ void init() {
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int q = 0; q < H; ++q)
#pragma unroll
        for (int r = 0; r < H; ++r) Eh[c][q][r] = El[c][q][r] = make_float2(0.f, 0.f);
    Eh[0][0][0].x = 1.f;
    L = 0;
  }

  __device__ __forceinline__ void site(const uint8_t* ra, const uint8_t* rb) {
    float2 Ef[2][H][H];
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int q = 0; q < H; ++q)
#pragma unroll
        for (int r = 0; r < H; ++r)
          Ef[c][q][r] = make_float2(__fadd_rn(Eh[c][q][r].x, El[c][q][r].x), __fadd_rn(Eh[c][q][r].y, El[c][q][r].y));
    float2 Nh[2][H][H], Nl[2][H][H];
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int p = 0; p < H; ++p)
#pragma unroll
        for (int r = 0; r < H; ++r) Nh[s][p][r] = Nl[s][p][r] = make_float2(0.f, 0.f);
#pragma unroll
    for (int s = 0; s < 2; ++s) {
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const uint8_t* pa = ra + (2 * c + s) * Rec::kBlockBytes;
        const uint8_t* pb = rb + (2 * c + s) * Rec::kBlockBytes;
        float2 ah[H][H], al[H][H], bh[H][H], bl[H][H];
        load_block_f<H>(pa, ah);
        load_block_f<H>(pa + H * H * 8, al);
        load_block_f<H>(pb, bh);
        load_block_f<H>(pb + H * H * 8, bl);
        // step 1: X[p][r] = sum_q a[q][p] E_c[q][r]
        float2 Xh[H][H], Xl[H][H];
#pragma unroll
        for (int p = 0; p < H; ++p) {
#pragma unroll
          for (int r = 0; r < H; ++r) {
            float hr = 0.f, hi = 0.f, lr = 0.f, li = 0.f;
#pragma unroll
            for (int q = 0; q < H; ++q) {
              const float2 A = ah[q][p], Al = al[q][p];
              const float2 e = Eh[c][q][r], el = El[c][q][r], ef = Ef[c][q][r];
              hr = __fmaf_rn(A.x, e.x, hr);
              hr = __fmaf_rn(-A.y, e.y, hr);
              hi = __fmaf_rn(A.x, e.y, hi);
              hi = __fmaf_rn(A.y, e.x, hi);
              lr = __fmaf_rn(A.x, el.x, lr);
              lr = __fmaf_rn(-A.y, el.y, lr);
              lr = __fmaf_rn(Al.x, ef.x, lr);
              lr = __fmaf_rn(-Al.y, ef.y, lr);
              li = __fmaf_rn(A.x, el.y, li);
              li = __fmaf_rn(A.y, el.x, li);
              li = __fmaf_rn(Al.x, ef.y, li);
              li = __fmaf_rn(Al.y, ef.x, li);
            }
            const float xr = grid_round<GX>(__fadd_rn(hr, lr));
            const float xi = grid_round<GX>(__fadd_rn(hi, li));
            Xh[p][r] = make_float2(xr, xi);
            Xl[p][r] = make_float2(__fadd_rn(__fsub_rn(hr, xr), lr), __fadd_rn(__fsub_rn(hi, xi), li));
          }
        }
        // step 2: N_s[p][pp] += sum_r X[p][r] conj(b[r][pp])
#pragma unroll
        for (int p = 0; p < H; ++p) {
#pragma unroll
          for (int pp = 0; pp < H; ++pp) {
            float hr = Nh[s][p][pp].x, hi = Nh[s][p][pp].y, lr = Nl[s][p][pp].x, li = Nl[s][p][pp].y;
#pragma unroll
            for (int r = 0; r < H; ++r) {
              const float2 X = Xh[p][r], Xo = Xl[p][r], B = bh[r][pp], Bl = bl[r][pp];
              const float2 Bf = make_float2(__fadd_rn(B.x, Bl.x), __fadd_rn(B.y, Bl.y));
              hr = __fmaf_rn(X.x, B.x, hr);
              hr = __fmaf_rn(X.y, B.y, hr);
              hi = __fmaf_rn(X.y, B.x, hi);
              hi = __fmaf_rn(-X.x, B.y, hi);
              lr = __fmaf_rn(X.x, Bl.x, lr);
              lr = __fmaf_rn(X.y, Bl.y, lr);
              lr = __fmaf_rn(Xo.x, Bf.x, lr);
              lr = __fmaf_rn(Xo.y, Bf.y, lr);
              li = __fmaf_rn(X.y, Bl.x, li);
              li = __fmaf_rn(-X.x, Bl.y, li);
              li = __fmaf_rn(Xo.y, Bf.x, li);
              li = __fmaf_rn(-Xo.x, Bf.y, li);
            }
            Nh[s][p][pp] = make_float2(hr, hi);
            Nl[s][p][pp] = make_float2(lr, li);
          }
        }
      }
    }
    // renormalise by 2^-e (max |component| into [0.5, 1)) and re-split onto the E grid
    float m = 0.f;
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int p = 0; p < H; ++p)
#pragma unroll
        for (int r = 0; r < H; ++r)
          m = fmaxf(m, fmaxf(fabsf(__fadd_rn(Nh[s][p][r].x, Nl[s][p][r].x)),
                             fabsf(__fadd_rn(Nh[s][p][r].y, Nl[s][p][r].y))));
    int e = 0;
    if (m > 0.f && isfinite(m)) {
      frexpf(m, &e);
      if (e < -120) {  // collapse to near zero: scale up in two exact steps
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
          for (int p = 0; p < H; ++p)
#pragma unroll
            for (int r = 0; r < H; ++r) {
              Nh[s][p][r].x *= pow2f(100);
              Nh[s][p][r].y *= pow2f(100);
              Nl[s][p][r].x *= pow2f(100);
              Nl[s][p][r].y *= pow2f(100);
            }
        L -= 100;
        e += 100;
      }
    }
    const float sc = pow2f(-e);
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int p = 0; p < H; ++p)
#pragma unroll
        for (int r = 0; r < H; ++r) {
          const float hs = __fmul_rn(Nh[s][p][r].x, sc), ls = __fmul_rn(Nl[s][p][r].x, sc);
          const float hs2 = __fmul_rn(Nh[s][p][r].y, sc), ls2 = __fmul_rn(Nl[s][p][r].y, sc);
          const float eh = grid_round<kGridE>(__fadd_rn(hs, ls));
          const float eh2 = grid_round<kGridE>(__fadd_rn(hs2, ls2));
          Eh[s][p][r] = make_float2(eh, eh2);
          El[s][p][r] = make_float2(__fadd_rn(__fsub_rn(hs, eh), ls), __fadd_rn(__fsub_rn(hs2, eh2), ls2));
        }
    L += e;
  }

  __device__ __forceinline__ void renorm() {}

  __device__ __forceinline__ void amplitude(double& re, double& im) const {
    re = ((double)Eh[0][0][0].x + (double)El[0][0][0].x) + ((double)Eh[1][0][0].x + (double)El[1][0][0].x);
    im = ((double)Eh[0][0][0].y + (double)El[0][0][0].y) + ((double)Eh[1][0][0].y + (double)El[1][0][0].y);
  }
};

// ------------------------------------------------------- tile kernel ------
// Device status word of this translation unit (QSVM_OK or QSVM_ERR_TIMEOUT).
__device__ int32_t g_pair_status;

// Upper-triangle tile index b (row-major, T tiles per side) -> (ti, tj), ti <= tj.
__device__ __forceinline__ void tri_decode(int64_t b, int64_t T, int64_t& ti, int64_t& tj) {
  const double tt = 2.0 * (double)T + 1.0;
  int64_t r = (int64_t)floor((tt - sqrt(tt * tt - 8.0 * (double)b)) * 0.5);
  if (r < 0) r = 0;
  if (r > T - 1) r = T - 1;
  // start(r) = r*T - r(r-1)/2 ; fix rounding
  while (r > 0 && r * T - r * (r - 1) / 2 > b) --r;
  while (r + 1 < T && (r + 1) * T - (r + 1) * r / 2 <= b) ++r;
  ti = r;
  tj = r + (b - (r * T - r * (r - 1) / 2));
}

template <int CHI, int PREC>
struct TileCfg {
  using Rec = Record<CHI, PREC>;
  static constexpr int TI = 16;                               // TI x TI pairs, one per thread
  static constexpr int S = (Rec::kBytes >= 1024) ? 1 : (1024 / Rec::kBytes);  // sites per chunk
  static constexpr int SLOT = S * Rec::kBytes + 16;           // +16 B: spreads points over banks
  static constexpr int STAGE = 2 * TI * SLOT;
  static constexpr int kOutBytes = TI * (TI + 1) * 16;
  static constexpr int kSmem = 2 * STAGE + kOutBytes + 64;
};

template <int CHI, int PREC>
__global__ void __launch_bounds__(256) pair_tile_kernel(TileArgs args) {
  using Cfg = TileCfg<CHI, PREC>;
  using Rec = Record<CHI, PREC>;
  constexpr int TI = Cfg::TI, S = Cfg::S, SLOT = Cfg::SLOT, STAGE = Cfg::STAGE;
  extern __shared__ __align__(128) uint8_t smem[];
  double* outK = reinterpret_cast<double*>(smem + 2 * STAGE);
  double* outL = outK + TI * (TI + 1);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + 2 * STAGE + Cfg::kOutBytes);

  const int64_t b = args.tile_begin + blockIdx.x;
  int64_t ti, tj;
  if (args.symmetric) {
    tri_decode(b, args.tiles_j, ti, tj);
  } else {
    ti = b / args.tiles_j;
    tj = b - ti * args.tiles_j;
  }
  const int64_t i0 = ti * TI, j0 = tj * TI;
  const int ni = (int)((args.nA - i0) < TI ? (args.nA - i0) : TI);
  const int nj = (int)((args.nB - j0) < TI ? (args.nB - j0) : TI);
  const int n = args.n;
  const int tid = threadIdx.x;
  const int ty = tid / TI, tx = tid % TI;
  const bool diag_tile = args.symmetric && ti == tj;
  const bool valid = ty < ni && tx < nj && (!diag_tile || ty <= tx);
  const int slotA = min(ty, ni - 1);
  const int slotB = TI + min(tx, nj - 1);
  const int nchunks = (n + S - 1) / S;

  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    fence_mbar_init();
  }
  __syncthreads();

  auto issue = [&](int ch, int st) {
    const int k0 = ch * S;
    const int ns = min(S, n - k0);
    const uint32_t bytes = (uint32_t)(ns * Rec::kBytes);
    mbar_arrive_expect_tx(&bars[st], bytes * (uint32_t)(ni + nj));
    uint8_t* base = smem + st * STAGE;
    for (int p = 0; p < ni; ++p)
      bulk_g2s(base + p * SLOT, args.mpsA + ((i0 + p) * (int64_t)n + k0) * Rec::kBytes, bytes, &bars[st]);
    for (int p = 0; p < nj; ++p)
      bulk_g2s(base + (TI + p) * SLOT, args.mpsB + ((j0 + p) * (int64_t)n + k0) * Rec::kBytes, bytes, &bars[st]);
  };

  if (tid == 0) {
    issue(0, 0);
    if (nchunks > 1) issue(1, 1);
  }

  Engine<CHI, PREC> eng;
  eng.init();
  int failed_chunk = -1;
  for (int ch = 0; ch < nchunks; ++ch) {
    const int st = ch & 1;
    const bool ok = mbar_wait_bounded(&bars[st], (uint32_t)((ch >> 1) & 1), kWaitLimitNs);
    if (__syncthreads_or(!ok)) {
      failed_chunk = ch;
      break;
    }
    const uint8_t* base = smem + st * STAGE;
    const int k0 = ch * S;
    const int ns = min(S, n - k0);
    if (valid) {
      const uint8_t* pa = base + slotA * SLOT;
      const uint8_t* pb = base + slotB * SLOT;
#pragma unroll 1
      for (int s = 0; s < ns; ++s) {
        eng.site(pa + s * Rec::kBytes, pb + s * Rec::kBytes);
        if (Engine<CHI, PREC>::kRenormEvery > 1 && ((k0 + s + 1) % Engine<CHI, PREC>::kRenormEvery) == 0)
          eng.renorm();
      }
    }
    __syncthreads();
    if (tid == 0 && ch + 2 < nchunks) issue(ch + 2, st);
  }

  if (failed_chunk >= 0) {
    // A copy never completed: record it, wait (bounded) for the copies this CTA
    // still has in flight, and leave without writing results.
    if (tid == 0) {
      atomicCAS(&g_pair_status, 0, (int32_t)QSVM_ERR_TIMEOUT);
      for (int ch = failed_chunk; ch < min(failed_chunk + 2, nchunks); ++ch)
        mbar_wait_bounded(&bars[ch & 1], (uint32_t)((ch >> 1) & 1), kDrainLimitNs);
    }
    return;
  }

  double kval = 0.0, lval = -INFINITY;
  if (valid) {
    if (Engine<CHI, PREC>::kRenormEvery > 1) eng.renorm();
    double re, im;
    eng.amplitude(re, im);
    const double a2 = re * re + im * im;
    if (a2 > 0.0) {
      kval = ldexp(a2, 2 * eng.L);
      lval = log(a2) + (double)(2 * eng.L) * 0.69314718055994530942;
    }
    args.K[(i0 + ty) * args.ldk + (j0 + tx)] = kval;
    if (args.logK) args.logK[(i0 + ty) * args.ldl + (j0 + tx)] = lval;
  }
  if (args.symmetric) {
    // mirror K[j][i] = K[i][j] bit-exactly, through shared memory so that the
    // transposed rows are written contiguously
    outK[ty * (TI + 1) + tx] = kval;
    outL[ty * (TI + 1) + tx] = lval;
    __syncthreads();
    // this thread writes row j0+ty, column i0+tx: the value of pair (i0+tx, j0+ty)
    const bool src = tx < ni && ty < nj && (!diag_tile || tx < ty);
    if (src) {
      args.K[(j0 + ty) * args.ldk + (i0 + tx)] = outK[tx * (TI + 1) + ty];
      if (args.logK) args.logK[(j0 + ty) * args.ldl + (i0 + tx)] = outL[tx * (TI + 1) + ty];
    }
  }
}

}  // namespace qsvm
