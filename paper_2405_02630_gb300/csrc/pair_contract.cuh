// pair_contract.cuh -- all-pairs transfer-matrix contraction (K3, FP32, split FP32).
//
// For a pair (i, j) the overlap <psi_j|psi_i> of arXiv 2405.02630 Eq. 4 is
// contracted along the chain (the tensor-network kernel of Algorithm 2, whose
// path is the fixed left-to-right order on a chain):
//     E_0 = e_0 e_0^T,   E_{k+1} = sum_sigma (A_{i,k}^sigma)^T E_k conj(A_{j,k}^sigma),
//     amp = trace(E_n)   (the last site's right bond carries sigma).
// The feature map ends on a diagonal layer, so A^sigma[t][u] vanishes unless the
// low bit of u equals sigma; E is then block diagonal in (t & 1, t' & 1) and the
// update splits into chi/2-sized blocks a_cs[q][p] = A^s[2q+c][2p+s]:
//     E'_s = sum_c a_cs^T E_c conj(b_cs).
// The low bit c of the left bond enters the site tensor only through the last
// repetition's ZZ phase, so a_1s = r_s a_0s with r_0 = exp(2 i theta_{k-1}) and
// r_1 = conj(r_0) (the record stores a_0s and r).  Hence
//     E'_s = a_0s^T (E_0 + rho_s E_1) conj(b_0s),   rho_s = r_s(i) conj(r_s(j)),
// chi^3/2 + chi^2/2 + 1 complex MACs per site instead of chi^3 (the block form,
// reps = 1).  Plain FP32 at reps = 2 generates the site tensors in registers from
// three unit phases per site (the phase form, 33 complex MACs per site).  FP64 and
// split FP32 at reps = 2 and 3 use the gauged form (a change of bond basis after
// which a site is two phases alpha, beta; see Record<4, QSVM_FP32_SPLIT>): 26
// complex MACs per site at reps = 2, 160 at reps = 3, plus one virtual site.
//
// One CTA owns a TI x TI tile of pairs, one thread per pair, E in registers for
// all n sites.  The tile's 2*TI points stream their site records through shared
// memory in chunks of S sites: one thread issues one bulk (TMA) copy per point
// and chunk, completion is tracked by an mbarrier per stage.
//
// Renormalisation: E is scaled by an exact power of two and the exponent is
// accumulated in an integer, so the scale is exact (the split reps = 2 engine lets
// its grids follow E's exponent and rescales every few sites instead).
#pragma once

#include <math.h>

#include "qsvm_common.cuh"

namespace qsvm {

// ---------------------------------------------------------- loads ---------
// Site records are addressed by 32-bit shared-window offsets and read through a
// __shared__-derived pointer, so the compiler emits LDS and can schedule them.
extern __shared__ __align__(128) uint8_t qsvm_dyn_smem[];

__device__ __forceinline__ const uint8_t* sptr(uint32_t a) {
  return qsvm_dyn_smem + (a - static_cast<uint32_t>(__cvta_generic_to_shared(qsvm_dyn_smem)));
}

template <int H>
__device__ __forceinline__ void load_block_d(uint32_t a, double2 (&d)[H][H]) {
  const double2* q = reinterpret_cast<const double2*>(sptr(a));
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

  __device__ __forceinline__ void site(uint32_t ra, uint32_t rb) {
    // rho_0 = r(i) conj(r(j)); rho_1 = conj(rho_0)
    const double2 ri = *reinterpret_cast<const double2*>(sptr(ra + Rec::kPhaseOff));
    const double2 rj = *reinterpret_cast<const double2*>(sptr(rb + Rec::kPhaseOff));
    const double pr = fma(ri.x, rj.x, ri.y * rj.y), pi = fma(ri.y, rj.x, -ri.x * rj.y);
    // G_s = E_0 + rho_s E_1, in place: with T = E_0 + Re(rho) E_1,
    // G_0 = T + Im(rho) i E_1 and G_1 = T - Im(rho) i E_1
#pragma unroll
    for (int q = 0; q < H; ++q)
#pragma unroll
      for (int r = 0; r < H; ++r) {
        const double2 e0 = E[0][q][r], e1 = E[1][q][r];
        const double tr = fma(pr, e1.x, e0.x), ti = fma(pr, e1.y, e0.y);
        E[0][q][r] = make_double2(fma(-pi, e1.y, tr), fma(pi, e1.x, ti));
        E[1][q][r] = make_double2(fma(pi, e1.y, tr), fma(-pi, e1.x, ti));
      }
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      double2 a[H][H], b[H][H];
      load_block_d<H>(ra + s * Rec::kBlockStride, a);
      load_block_d<H>(rb + s * Rec::kBlockStride, b);
      double2 X[H][H];
#pragma unroll
      for (int p = 0; p < H; ++p)
#pragma unroll
        for (int r = 0; r < H; ++r) {  // X[p][r] = sum_q a[q][p] G_s[q][r]
          double xr = 0.0, xi = 0.0;
#pragma unroll
          for (int q = 0; q < H; ++q) {
            const double2 A = a[q][p], g = E[s][q][r];
            xr = fma(A.x, g.x, xr);
            xr = fma(-A.y, g.y, xr);
            xi = fma(A.x, g.y, xi);
            xi = fma(A.y, g.x, xi);
          }
          X[p][r] = make_double2(xr, xi);
        }
#pragma unroll
      for (int p = 0; p < H; ++p)
#pragma unroll
        for (int pp = 0; pp < H; ++pp) {  // E'_s[p][pp] = sum_r X[p][r] conj(b[r][pp])
          double nr = 0.0, ni = 0.0;
#pragma unroll
          for (int r = 0; r < H; ++r) {
            const double2 B = b[r][pp];
            nr = fma(X[p][r].x, B.x, nr);
            nr = fma(X[p][r].y, B.y, nr);
            ni = fma(X[p][r].y, B.x, ni);
            ni = fma(-X[p][r].x, B.y, ni);
          }
          E[s][p][pp] = make_double2(nr, ni);
        }
    }
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
    re = __dadd_rn(E[0][0][0].x, E[1][0][0].x);
    im = __dadd_rn(E[0][0][0].y, E[1][0][0].y);
  }
};

// ------------------------------------------------------ packed FP32 ---------
// FP32x2 operations (one instruction, two lanes, each lane rounded exactly like
// the scalar __fmaf_rn / __fadd_rn / __fmul_rn).
__device__ __forceinline__ float2 bc(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
template <int G>
__device__ __forceinline__ float2 grid_round2(float2 v) {
  constexpr float C = 1.5f * (float)(1 << (23 - G));
  return add2(add2(v, make_float2(C, C)), make_float2(-C, -C));
}

// The frexp exponent of a positive float: m in [2^(e-1), 2^e) for normal m; -126
// for subnormal m (whose callers rescale in an extra exact step).
__device__ __forceinline__ int exp_of(float m) { return (int)((__float_as_uint(m) >> 23) & 0xffu) - 126; }

// Largest |component| of n packed values, as a tree (n a power of two).
template <int NV>
__device__ __forceinline__ float max_abs(const float2 (&v)[NV]) {
  float t[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) t[i] = fmaxf(fabsf(v[i].x), fabsf(v[i].y));
#pragma unroll
  for (int w = NV / 2; w >= 1; w >>= 1)
#pragma unroll
    for (int i = 0; i < w; ++i) t[i] = fmaxf(t[i], t[i + w]);
  return t[0];
}

// A block of form entries: first pair (A or conj B), second pair (iA or i conj B).
template <int H>
__device__ __forceinline__ void load_forms(uint32_t a, float2 (&x)[H][H], float2 (&ix)[H][H]) {
  const float4* q = reinterpret_cast<const float4*>(sptr(a));
#pragma unroll
  for (int e = 0; e < H * H; ++e) {
    const float4 v = q[e];
    x[e / H][e % H] = make_float2(v.x, v.y);
    ix[e / H][e % H] = make_float2(v.z, v.w);
  }
}

// Plain FP32: complex values as (re, im) lane pairs; a complex MAC is two
// packed FMAs, E A = E.re (A) + E.im (iA) and X conj(B) = X.re (conj B) +
// X.im (i conj B), with the tensor side read ready-made from the two record
// forms.  Renormalised every 4 sites.
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

  __device__ __forceinline__ void site(uint32_t ra, uint32_t rb) {
    // rho_0 = r(i) conj(r(j)) from r(i)'s a-form components and r(j)'s b-form pair
    const float4 fi = *reinterpret_cast<const float4*>(sptr(ra + Rec::kPhaseOff));
    const float4 fj = *reinterpret_cast<const float4*>(sptr(rb + Rec::kPhaseOff));
    const float2 rho = fma2(bc(fi.x), make_float2(fj.x, fj.y), mul2(bc(fi.y), make_float2(fj.z, fj.w)));
    // forms: rho_0 = (a, b), i rho_0 = (-b, a); rho_1 = (a, -b), i rho_1 = (b, a)
    const float2 R0 = rho, iR0 = make_float2(-rho.y, rho.x);
    const float2 R1 = make_float2(rho.x, -rho.y), iR1 = make_float2(rho.y, rho.x);
    // G_s = E_0 + rho_s E_1 = E_0 + E_1.re (rho_s) + E_1.im (i rho_s), in place
#pragma unroll
    for (int q = 0; q < H; ++q)
#pragma unroll
      for (int r = 0; r < H; ++r) {
        const float2 e0 = E[0][q][r], e1 = E[1][q][r];
        E[0][q][r] = fma2(bc(e1.y), iR0, fma2(bc(e1.x), R0, e0));
        E[1][q][r] = fma2(bc(e1.y), iR1, fma2(bc(e1.x), R1, e0));
      }
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      float2 A[H][H], iA[H][H], cB[H][H], icB[H][H];
      load_forms<H>(ra + s * Rec::kBlockStride, A, iA);
      load_forms<H>(rb + s * Rec::kBlockStride, cB, icB);
      float2 X[H][H];
#pragma unroll
      for (int p = 0; p < H; ++p)
#pragma unroll
        for (int r = 0; r < H; ++r) {  // X[p][r] = sum_q a[q][p] G_s[q][r]
          float2 x = make_float2(0.f, 0.f);
#pragma unroll
          for (int q = 0; q < H; ++q) {
            x = fma2(bc(E[s][q][r].x), A[q][p], x);
            x = fma2(bc(E[s][q][r].y), iA[q][p], x);
          }
          X[p][r] = x;
        }
#pragma unroll
      for (int p = 0; p < H; ++p)
#pragma unroll
        for (int pp = 0; pp < H; ++pp) {  // E'_s[p][pp] = sum_r X[p][r] conj(b[r][pp])
          float2 acc = make_float2(0.f, 0.f);
#pragma unroll
          for (int r = 0; r < H; ++r) {
            acc = fma2(bc(X[p][r].x), cB[r][pp], acc);
            acc = fma2(bc(X[p][r].y), icB[r][pp], acc);
          }
          E[s][p][pp] = acc;
        }
    }
  }

  __device__ __forceinline__ void renorm() {
    const float m = max_abs<2 * H * H>(reinterpret_cast<const float2(&)[2 * H * H]>(E));
    if (!(m > 0.f) || !isfinite(m)) return;
    int e = exp_of(m);
    if (e < -120) {  // subnormal territory: scale in two exact steps
#pragma unroll
      for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int p = 0; p < H; ++p)
#pragma unroll
          for (int r = 0; r < H; ++r) E[s][p][r] = mul2(E[s][p][r], bc(pow2f(100)));
      L -= 100;
      e += 100;
    }
    const float2 sc = bc(pow2f(-e));
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int p = 0; p < H; ++p)
#pragma unroll
        for (int r = 0; r < H; ++r) E[s][p][r] = mul2(E[s][p][r], sc);
    L += e;
  }

  __device__ __forceinline__ void amplitude(double& re, double& im) const {
    re = __dadd_rn((double)E[0][0][0].x, (double)E[1][0][0].x);
    im = __dadd_rn((double)E[0][0][0].y, (double)E[1][0][0].y);
  }
};

// Split FP32.  Every value v is carried as hi + lo: hi on a fixed binary grid,
// lo the FP32 remainder.  Products of hi parts and their short sums are exact
// in FP32 FMAs because they stay on a common grid below 2^24 units (R = reps,
// H = chi/2; |a|, |b| = 2^{-R/2}, |r| = 1; E renormalised to components <= 1):
//   rho = r(i) conj(r(j)):  hi(r) on 2^-11, two products  ->  <= 2^23 units of 2^-22;
//   G = E_0 + rho E_1:      hi(E) on 2^-10, hi(rho) on 2^-11, three terms
//                           ->  < 3 * 2^21 units of 2^-21;  |G| <= 1 + sqrt(2);
//   X = a^T G:              hi(G) on 2^-10, hi(a) on 2^-11, 2H products
//                           ->  <= 1.44e7 units of 2^-21 (chi = 8; 1.0e7 for chi = 4);
//   E' = X conj(b):         |X| <= H 2^{-R/2} 2 sqrt(2), hi(X) on 2^-GX (GX = 10, or
//                           9 for chi = 8), 2H products  ->  < 1.19e7 units of 2^-(GX+11)
//   (2^24 = 1.68e7).
// The remaining terms use u = hi(u) + lo(u):
//   u w = hi(u) hi(w) + hi(u) lo(w) + lo(u) full(w)
// where full() is the rounded FP32 sum hi + lo.  Each correction is about 2^-11
// of the result, so its FP32 rounding costs ~2^-35 relative per step; nothing
// else is rounded.  This is the split hi+lo compensated product carried out on
// the FP32 pipe: 6 packed FMAs (12 FMAs) per complex MAC.

// rho = u conj(w) for split values given as u's a-form entries (hi at ah, lo at al)
// and w's b-form entries (hi at bh, lo at bl), returned as the split forms R = rho,
// iR = i rho; hi(rho) on 2^-kGridT.
__device__ __forceinline__ void split_rho(uint32_t ah, uint32_t al, uint32_t bh, uint32_t bl, float2& Rh, float2& iRh,
                                          float2& Rl, float2& iRl) {
  const float4 ih = *reinterpret_cast<const float4*>(sptr(ah));
  const float4 il = *reinterpret_cast<const float4*>(sptr(al));
  const float4 jh = *reinterpret_cast<const float4*>(sptr(bh));
  const float4 jl = *reinterpret_cast<const float4*>(sptr(bl));
  const float2 cjh = make_float2(jh.x, jh.y), icjh = make_float2(jh.z, jh.w);
  const float2 cjl = make_float2(jl.x, jl.y), icjl = make_float2(jl.z, jl.w);
  const float2 h = fma2(bc(ih.x), cjh, mul2(bc(ih.y), icjh));  // exact
  const float fx = ih.x + il.x, fy = ih.y + il.y;
  const float2 l = fma2(bc(il.x), cjh, fma2(bc(il.y), icjh, fma2(bc(fx), cjl, mul2(bc(fy), icjl))));
  const float2 v = add2(h, l);
  const float2 rh = grid_round2<kGridT>(v);
  const float2 rl = add2(fma2(rh, make_float2(-1.f, -1.f), h), l);  // (h - rh) is exact
  Rh = rh;
  iRh = make_float2(-rh.y, rh.x);
  Rl = rl;
  iRl = make_float2(-rl.y, rl.x);
}

// As split_rho, also returning the forms of rho_1 = conj(rho_0): R[s] = rho_s, iR[s] = i rho_s.
__device__ __forceinline__ void split_phase(uint32_t ah, uint32_t al, uint32_t bh, uint32_t bl, float2 (&Rh)[2],
                                            float2 (&iRh)[2], float2 (&Rl)[2], float2 (&iRl)[2]) {
  split_rho(ah, al, bh, bl, Rh[0], iRh[0], Rl[0], iRl[0]);
  Rh[1] = make_float2(Rh[0].x, -Rh[0].y);
  iRh[1] = make_float2(Rh[0].y, Rh[0].x);
  Rl[1] = make_float2(Rl[0].x, -Rl[0].y);
  iRl[1] = make_float2(Rl[0].y, Rl[0].x);
}

// G = E_0 + rho E_1 split onto the 2^-GG grid (hi, lo, full).
template <int GG = kGridG>
__device__ __forceinline__ void split_mix(float2 e0h, float2 e0l, float2 e1h, float2 e1l, float2 e1f, float2 Rh,
                                          float2 iRh, float2 Rl, float2 iRl, float2& gh, float2& gl, float2& gf) {
  const float2 h = fma2(bc(e1h.y), iRh, fma2(bc(e1h.x), Rh, e0h));  // exact
  const float2 l = fma2(bc(e1f.y), iRl, fma2(bc(e1f.x), Rl, fma2(bc(e1l.y), iRh, fma2(bc(e1l.x), Rh, e0l))));
  const float2 v = add2(h, l);
  gh = grid_round2<GG>(v);
  gl = add2(fma2(gh, make_float2(-1.f, -1.f), h), l);  // (h - gh) is exact
  gf = v;
}

template <int CHI>
struct Engine<CHI, QSVM_FP32_SPLIT> {
  static constexpr int H = CHI / 2;
  static constexpr int GX = grid_x(CHI);
  static constexpr int kRenormEvery = 1;  // built into site()
  using Rec = Record<CHI, QSVM_FP32_SPLIT>;
  float2 Eh[2][H][H], El[2][H][H], Ef[2][H][H];  // Ef = fl(Eh + El)
  int L;

  __device__ __forceinline__ void init() {
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int q = 0; q < H; ++q)
#pragma unroll
        for (int r = 0; r < H; ++r) Eh[c][q][r] = El[c][q][r] = Ef[c][q][r] = make_float2(0.f, 0.f);
    Eh[0][0][0].x = Ef[0][0][0].x = 1.f;
    L = 0;
  }

  __device__ __forceinline__ void site(uint32_t ra, uint32_t rb) {
    const float2 m1 = make_float2(-1.f, -1.f);
    float2 Rh[2], iRh[2], Rl[2], iRl[2];
    split_phase(ra + Rec::kPhaseOff, ra + Rec::kPhaseOff + 16, rb + Rec::kPhaseOff, rb + Rec::kPhaseOff + 16, Rh, iRh,
                Rl, iRl);
    // G_s = E_0 + rho_s E_1, in place of E_s
#pragma unroll
    for (int q = 0; q < H; ++q)
#pragma unroll
      for (int r = 0; r < H; ++r) {
        const float2 e0h = Eh[0][q][r], e0l = El[0][q][r];
        const float2 e1h = Eh[1][q][r], e1l = El[1][q][r], e1f = Ef[1][q][r];
#pragma unroll
        for (int s = 0; s < 2; ++s)
          split_mix(e0h, e0l, e1h, e1l, e1f, Rh[s], iRh[s], Rl[s], iRl[s], Eh[s][q][r], El[s][q][r], Ef[s][q][r]);
      }
    float2 Nh[2][H][H], Nl[2][H][H];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const uint32_t pa = ra + s * Rec::kBlockStride;
      const uint32_t pb = rb + s * Rec::kBlockStride;
      float2 Ah[H][H], iAh[H][H], Al[H][H], iAl[H][H];
      float2 Bh[H][H], iBh[H][H], Bl[H][H], iBl[H][H];  // conj(b) and i conj(b), hi and lo
      load_forms<H>(pa, Ah, iAh);
      load_forms<H>(pa + Rec::kPartBytes, Al, iAl);
      load_forms<H>(pb, Bh, iBh);
      load_forms<H>(pb + Rec::kPartBytes, Bl, iBl);
      // X[p][r] = sum_q a[q][p] G_s[q][r]
      float2 Xh[H][H], Xl[H][H], Xf[H][H];
#pragma unroll
      for (int p = 0; p < H; ++p) {
#pragma unroll
        for (int r = 0; r < H; ++r) {
          float2 h = make_float2(0.f, 0.f), l = make_float2(0.f, 0.f);
#pragma unroll
          for (int q = 0; q < H; ++q) {
            const float2 g = Eh[s][q][r], gl = El[s][q][r], gf = Ef[s][q][r];
            h = fma2(bc(g.x), Ah[q][p], h);
            h = fma2(bc(g.y), iAh[q][p], h);
            l = fma2(bc(gl.x), Ah[q][p], l);
            l = fma2(bc(gl.y), iAh[q][p], l);
            l = fma2(bc(gf.x), Al[q][p], l);
            l = fma2(bc(gf.y), iAl[q][p], l);
          }
          const float2 v = add2(h, l);
          const float2 xh = grid_round2<GX>(v);
          Xh[p][r] = xh;
          Xl[p][r] = add2(fma2(xh, m1, h), l);  // (h - xh) is exact
          Xf[p][r] = v;
        }
      }
      // E'_s[p][pp] = sum_r X[p][r] conj(b[r][pp])
#pragma unroll
      for (int p = 0; p < H; ++p) {
#pragma unroll
        for (int pp = 0; pp < H; ++pp) {
          float2 hh = make_float2(0.f, 0.f), ll = make_float2(0.f, 0.f);
#pragma unroll
          for (int r = 0; r < H; ++r) {
            const float2 xh = Xh[p][r], xl = Xl[p][r], xf = Xf[p][r];
            hh = fma2(bc(xh.x), Bh[r][pp], hh);
            hh = fma2(bc(xh.y), iBh[r][pp], hh);
            ll = fma2(bc(xf.x), Bl[r][pp], ll);
            ll = fma2(bc(xf.y), iBl[r][pp], ll);
            ll = fma2(bc(xl.x), Bh[r][pp], ll);
            ll = fma2(bc(xl.y), iBh[r][pp], ll);
          }
          Nh[s][p][pp] = hh;
          Nl[s][p][pp] = ll;
        }
      }
    }
    // renormalise by 2^-e (max |component| of hi + lo into [0.5, 1)) and re-split onto the E grid
    float2 V[2][H][H];
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int p = 0; p < H; ++p)
#pragma unroll
        for (int r = 0; r < H; ++r) V[s][p][r] = add2(Nh[s][p][r], Nl[s][p][r]);
    const float m = max_abs<2 * H * H>(reinterpret_cast<const float2(&)[2 * H * H]>(V));
    int e = 0;
    if (m > 0.f && isfinite(m)) {
      e = exp_of(m);
      if (e < -120) {  // collapse to near zero: scale up in two exact steps
        const float2 up = bc(pow2f(100));
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
          for (int p = 0; p < H; ++p)
#pragma unroll
            for (int r = 0; r < H; ++r) {
              Nh[s][p][r] = mul2(Nh[s][p][r], up);
              Nl[s][p][r] = mul2(Nl[s][p][r], up);
              V[s][p][r] = mul2(V[s][p][r], up);
            }
        L -= 100;
        e += 100;
      }
    }
    const float2 sc = bc(pow2f(-e));
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int p = 0; p < H; ++p)
#pragma unroll
        for (int r = 0; r < H; ++r) {
          // full = (Nh + Nl) 2^-e; hi = grid(full); lo = (Nh 2^-e - hi) + Nl 2^-e, where
          // Nh 2^-e - hi is exact (both on grids whose difference fits in 24 bits)
          const float2 f = mul2(V[s][p][r], sc);
          const float2 h = grid_round2<kGridE>(f);
          Eh[s][p][r] = h;
          El[s][p][r] = fma2(Nl[s][p][r], sc, fma2(h, m1, mul2(Nh[s][p][r], sc)));
          Ef[s][p][r] = f;
        }
    L += e;
  }

  __device__ __forceinline__ void renorm() {}

  __device__ __forceinline__ void amplitude(double& re, double& im) const {
    re = __dadd_rn(__dadd_rn((double)Eh[0][0][0].x, (double)El[0][0][0].x),
                   __dadd_rn((double)Eh[1][0][0].x, (double)El[1][0][0].x));
    im = __dadd_rn(__dadd_rn((double)Eh[0][0][0].y, (double)El[0][0][0].y),
                   __dadd_rn((double)Eh[1][0][0].y, (double)El[1][0][0].y));
  }
};

// --------------------------------------- phase form (reps = 2, plain FP32) ----
// The row point's blocks, unscaled (their factors 1/2 go to the log scale:
// L -= 2 per site), with V0 = T^2, V1 = P^2, V2 = P^2 T^2 (rows q, columns p):
//   a_00 = [[V2, 1], [V1, V0]],   a_01 = [[1, -conj(V2)], [conj(V0), -conj(V1)]].
// The column point's phases are W0, W1, W2.  Per site:
//   rho_0 = W0 conj(V0) (= r(i) conj(r(j)) with r = conj(T^2)),  rho_1 = conj(rho_0),
//   G_s = E_0 + rho_s E_1;
//   s = 0:  X[0][r] = V2 G[0][r] + V1 G[1][r],      X[1][r] = G[0][r] + V0 G[1][r],
//           E'[p][0] = X[p][0] conj(W2) + X[p][1] conj(W1),   E'[p][1] = X[p][0] + X[p][1] conj(W0);
//   s = 1:  X[0][r] = G[0][r] + conj(V0) G[1][r],   X~[1][r] = conj(V2) G[0][r] + conj(V1) G[1][r],
//           E~[p][0] = X[p][0] + X[p][1] W0,        E~[p][1] = X[p][0] W2 + X[p][1] W1,
//           and since row 1 of X and column 1 of conj(b_01) carry a minus sign,
//           E'_1[p][pp] = (-1)^{p+pp} E~[p][pp].
// That is 33 complex MACs per site (chi^3/2 + chi^2/2 + 1 = 41 in the block
// form).  The last site keeps its right bond open, so amp = sum of all entries.

__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 zfma(double2 a, double2 b, double2 c) {  // a b + c
  return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}
__device__ __forceinline__ double2 zconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 zneg(double2 a) { return make_double2(-a.x, -a.y); }

template <>
struct Engine<4, QSVM_FP64> {
  // Gauged form (the records of split FP32 at reps = 2, in doubles): per site
  // Y_c[p][r] = E_c[0][r] + a[p] E_c[1][r] (a = (alpha_i, beta_i), E_1 stored with the
  // signs of S E_1 S), X_s = Y_0 + rho_s Y_1 (rho_0 = alpha_i conj(alpha_j), rho_1 =
  // beta_i conj(beta_j)), E'_s[p][pp] = X_s[p][0] + conj(b[pp]) X_s[p][1]: 24 complex MACs
  // and two phase products per site; the amplitude is E_0[0][0] after the virtual site.
  static constexpr int kRenormEvery = 8;
  using Rec = Record<4, QSVM_FP64>;
  double2 E[2][2][2];
  int L;

  __device__ __forceinline__ void init() {
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int r = 0; r < 2; ++r) E[c][q][r] = make_double2(0.0, 0.0);
    E[0][0][0].x = 1.0;
    L = 2;  // every site() counts -2 for the factors 1/2 of a and b; the virtual site has none
  }

  __device__ __forceinline__ void site(uint32_t ra, uint32_t rb) {
    const double2* a = reinterpret_cast<const double2*>(sptr(ra));
    const double2* b = reinterpret_cast<const double2*>(sptr(rb));
    const double2 A[2] = {a[0], a[1]};
    const double2 Bc[2] = {zconj(b[0]), zconj(b[1])};
    const double2 rho[2] = {zmul(A[0], Bc[0]), zmul(A[1], Bc[1])};
    double2 Y[2][2][2];
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int p = 0; p < 2; ++p)
#pragma unroll
        for (int r = 0; r < 2; ++r) Y[c][p][r] = zfma(A[p], E[c][1][r], E[c][0][r]);
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        const double2 x0 = zfma(rho[s], Y[1][p][0], Y[0][p][0]);
        const double2 x1 = zfma(rho[s], Y[1][p][1], Y[0][p][1]);
#pragma unroll
        for (int pp = 0; pp < 2; ++pp) {
          const double2 v = zfma(Bc[pp], x1, x0);
          E[s][p][pp] = (s == 1 && ((p + pp) & 1)) ? zneg(v) : v;
        }
      }
    L -= 2;
  }

  __device__ __forceinline__ void renorm() {
    double m = 0.0;
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int p = 0; p < 2; ++p)
#pragma unroll
        for (int r = 0; r < 2; ++r) m = fmax(m, fmax(fabs(E[s][p][r].x), fabs(E[s][p][r].y)));
    if (!(m > 0.0) || !isfinite(m)) return;
    int e;
    frexp(m, &e);
    if (e < -1000) e = -1000;
    const double sc = ldexp(1.0, -e);
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int p = 0; p < 2; ++p)
#pragma unroll
        for (int r = 0; r < 2; ++r) {
          E[s][p][r].x *= sc;
          E[s][p][r].y *= sc;
        }
    L += e;
  }

  // after the virtual site the amplitude is entry (0, 0) of block 0 (up to a phase)
  __device__ __forceinline__ void amplitude(double& re, double& im) const {
    re = E[0][0][0].x;
    im = E[0][0][0].y;
  }
};

template <>
struct Engine<8, QSVM_FP64> {
  // Gauged form at reps = 3 (the records of reps = 2, in doubles): both blocks of a site
  // are the signed Kronecker square of M = [[1, 1], [alpha, beta]] and block c = 1 adds
  // r'_s diag(1, 1, -1, -1); with the row signs T = diag(1, 1, 1, -1) and the S signs
  // folded into the stored environment, a site is Y_c = (M_i x M_i)^T E_c (two 2 x 2
  // stages over the row bits), X_s = Y_0 + rho_s Y_1, E'_s = X_s conj(M_j x M_j) (two
  // stages over the column bits): 160 complex MACs and two phase products.  Each stage
  // works in place on columns, entries or rows of the environment, all in registers.
  static constexpr int kRenormEvery = 8;
  using Rec = Record<8, QSVM_FP64>;
  double2 E[2][4][4];  // [c][q][r], q = q1 + 2 q2 (q1 the first layer)
  int L;

  __device__ __forceinline__ void init() {
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int r = 0; r < 4; ++r) E[c][q][r] = make_double2(0.0, 0.0);
    E[0][0][0].x = 1.0;
    L = 3;  // every site() counts -3 for the factors 2^{-3/2} of a and b; the virtual site has none
  }

  __device__ __forceinline__ void site(uint32_t ra, uint32_t rb) {
    const double2* a = reinterpret_cast<const double2*>(sptr(ra));
    const double2* b = reinterpret_cast<const double2*>(sptr(rb));
    const double2 A[2] = {a[0], a[1]};
    const double2 Bc[2] = {zconj(b[0]), zconj(b[1])};
    const double2 rho[2] = {zmul(A[0], Bc[0]), zmul(A[1], Bc[1])};
    // rows: Z[p1 + 2 q2] = E[2 q2] + M[p1] E[1 + 2 q2], then Y[p1 + 2 p2] = Z[p1] + M[p2] Z[p1 + 2]
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const double2 z0 = zfma(A[0], E[c][1][r], E[c][0][r]), z1 = zfma(A[1], E[c][1][r], E[c][0][r]);
        const double2 z2 = zfma(A[0], E[c][3][r], E[c][2][r]), z3 = zfma(A[1], E[c][3][r], E[c][2][r]);
        E[c][0][r] = zfma(A[0], z2, z0);
        E[c][1][r] = zfma(A[0], z3, z1);
        E[c][2][r] = zfma(A[1], z2, z0);
        E[c][3][r] = zfma(A[1], z3, z1);
      }
    // mix: X_s = Y_0 + rho_s Y_1
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const double2 y0 = E[0][p][r], y1 = E[1][p][r];
        E[0][p][r] = zfma(rho[0], y1, y0);
        E[1][p][r] = zfma(rho[1], y1, y0);
      }
    // columns: W[pp1 + 2 r2] = X[2 r2] + conj(M[pp1]) X[1 + 2 r2], then
    // E'[pp1 + 2 pp2] = W[pp1] + conj(M[pp2]) W[pp1 + 2]; the signs T S^s . S^s T
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        const double2 w0 = zfma(Bc[0], E[s][p][1], E[s][p][0]), w1 = zfma(Bc[1], E[s][p][1], E[s][p][0]);
        const double2 w2 = zfma(Bc[0], E[s][p][3], E[s][p][2]), w3 = zfma(Bc[1], E[s][p][3], E[s][p][2]);
        const double2 nv[4] = {zfma(Bc[0], w2, w0), zfma(Bc[0], w3, w1), zfma(Bc[1], w2, w0), zfma(Bc[1], w3, w1)};
#pragma unroll
        for (int pp = 0; pp < 4; ++pp) {
          const int neg = ((p == 3) ^ (pp == 3) ^ (s & ((p >> 1) ^ (pp >> 1)))) & 1;
          E[s][p][pp] = neg ? zneg(nv[pp]) : nv[pp];
        }
      }
    L -= 3;
  }

  __device__ __forceinline__ void renorm() {
    double m = 0.0;
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int r = 0; r < 4; ++r) m = fmax(m, fmax(fabs(E[c][q][r].x), fabs(E[c][q][r].y)));
    if (!(m > 0.0) || !isfinite(m)) return;
    int e;
    frexp(m, &e);
    if (e < -1000) e = -1000;
    const double sc = ldexp(1.0, -e);
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          E[c][q][r].x *= sc;
          E[c][q][r].y *= sc;
        }
    L += e;
  }

  // after the virtual site the amplitude is entry (0, 0) of block 0 (up to a phase)
  __device__ __forceinline__ void amplitude(double& re, double& im) const {
    re = E[0][0][0].x;
    im = E[0][0][0].y;
  }
};

// Form pair (V, iV) (f = 0) or (conj V, i conj V) (f = 1) of phase v of an FP32 record.
__device__ __forceinline__ void phase_form(uint32_t rec, int v, int f, float2& x, float2& ix) {
  const float4 q = *reinterpret_cast<const float4*>(sptr(rec + Record<4, QSVM_FP32>::off(v, f)));
  x = make_float2(q.x, q.y);
  ix = make_float2(q.z, q.w);
}
// w V + acc, for w broadcast and V given by its form pair
__device__ __forceinline__ float2 cmac(float2 w, float2 x, float2 ix, float2 acc) {
  return fma2(bc(w.y), ix, fma2(bc(w.x), x, acc));
}
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

template <>
struct Engine<4, QSVM_FP32> {
  static constexpr int kRenormEvery = 4;
  using Rec = Record<4, QSVM_FP32>;
  float2 E[2][2][2];
  int L;

  __device__ __forceinline__ void init() {
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int r = 0; r < 2; ++r) E[c][q][r] = make_float2(0.f, 0.f);
    E[0][0][0].x = 1.f;
    L = 0;
  }

  __device__ __forceinline__ void site(uint32_t ra, uint32_t rb) {
    const float2 z = make_float2(0.f, 0.f);
    float2 x0, ix0, x1, ix1, x2, ix2;
    // rho_0 = W0 conj(V0)
    phase_form(rb, 0, 0, x0, ix0);
    phase_form(ra, 0, 1, x1, ix1);
    const float2 r0 = cmac(x0, x1, ix1, z);
    const float2 R0 = r0, iR0 = make_float2(-r0.y, r0.x), R1 = make_float2(r0.x, -r0.y), iR1 = make_float2(r0.y, r0.x);
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const float2 e0 = E[0][q][r], e1 = E[1][q][r];
        E[0][q][r] = cmac(e1, R0, iR0, e0);
        E[1][q][r] = cmac(e1, R1, iR1, e0);
      }
    float2 X[2][2];
    // s = 0: row phases in a-form, column phases in b-form
    phase_form(ra, 0, 0, x0, ix0);
    phase_form(ra, 1, 0, x1, ix1);
    phase_form(ra, 2, 0, x2, ix2);
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      X[0][r] = cmac(E[0][1][r], x1, ix1, cmac(E[0][0][r], x2, ix2, z));
      X[1][r] = cmac(E[0][1][r], x0, ix0, E[0][0][r]);
    }
    phase_form(rb, 0, 1, x0, ix0);
    phase_form(rb, 1, 1, x1, ix1);
    phase_form(rb, 2, 1, x2, ix2);
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      E[0][p][0] = cmac(X[p][1], x1, ix1, cmac(X[p][0], x2, ix2, z));
      E[0][p][1] = cmac(X[p][1], x0, ix0, X[p][0]);
    }
    // s = 1: row phases in b-form, column phases in a-form
    phase_form(ra, 0, 1, x0, ix0);
    phase_form(ra, 1, 1, x1, ix1);
    phase_form(ra, 2, 1, x2, ix2);
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      X[0][r] = cmac(E[1][1][r], x0, ix0, E[1][0][r]);
      X[1][r] = cmac(E[1][1][r], x1, ix1, cmac(E[1][0][r], x2, ix2, z));  // X~[1][r]
    }
    phase_form(rb, 0, 0, x0, ix0);
    phase_form(rb, 1, 0, x1, ix1);
    phase_form(rb, 2, 0, x2, ix2);
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      const float2 n0 = cmac(X[p][1], x0, ix0, X[p][0]);
      const float2 n1 = cmac(X[p][1], x1, ix1, cmac(X[p][0], x2, ix2, z));
      E[1][p][0] = p ? neg2(n0) : n0;
      E[1][p][1] = p ? n1 : neg2(n1);
    }
    L -= 2;
  }

  __device__ __forceinline__ void renorm() {
    const float m = max_abs<8>(reinterpret_cast<const float2(&)[8]>(E));
    if (!(m > 0.f) || !isfinite(m)) return;
    int e = exp_of(m);
    if (e < -120) {  // subnormal territory: scale in two exact steps
#pragma unroll
      for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int p = 0; p < 2; ++p)
#pragma unroll
          for (int r = 0; r < 2; ++r) E[s][p][r] = mul2(E[s][p][r], bc(pow2f(100)));
      L -= 100;
      e += 100;
    }
    const float2 sc = bc(pow2f(-e));
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int p = 0; p < 2; ++p)
#pragma unroll
        for (int r = 0; r < 2; ++r) E[s][p][r] = mul2(E[s][p][r], sc);
    L += e;
  }

  __device__ __forceinline__ void amplitude(double& re, double& im) const {
    re = 0.0;
    im = 0.0;
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int p = 0; p < 2; ++p)
#pragma unroll
        for (int r = 0; r < 2; ++r) {
          re = __dadd_rn(re, (double)E[s][p][r].x);
          im = __dadd_rn(im, (double)E[s][p][r].y);
        }
  }
};

// ------------------------------------------- gauged form, split FP32 -----
// A split value's packed forms as read from a gauged-form record or formed for rho:
// hi (h, ih) and lo (l, il), each as the pair (V, iV) (row side, a-form) or
// (conj V, i conj V) (column side, b-form).
struct SplitForm {
  float2 h, ih, l, il;
};

template <>
struct Engine<4, QSVM_FP32_SPLIT> {
  // Gauged form: both blocks of a site are [[1, 1], [alpha, beta]] (row point) and
  // conj of the column point's, block c = 1 adds the factor r'_s S (S = diag(1, -1)).
  // Per site: Y_c[p][r] = E_c[0][r] + a[p] E_c[1][r] (a = (alpha_i, beta_i); E_1 is
  // stored with the signs of S E_1 S applied), shared by both s; X_s = Y_0 + rho_s Y_1
  // with rho_0 = alpha_i conj(alpha_j), rho_1 = beta_i conj(beta_j); E'_s[p][pp] =
  // X_s[p][0] + X_s[p][1] conj(b[pp]) (b = (alpha_j, beta_j)): 24 complex MACs and two
  // phase products per site, and 16 re-splits (Y_1, X[.][1], E; Y_0 and X[.][0] only
  // seed the next sum).  E is not rescaled every site: with U = 2^(e+1), e the frexp
  // exponent of E's largest component, E's components are below U/2 and the hi parts of
  // E, Y_1 and X[.][1] all sit on the grid U 2^-10 (one rounding constant per site, Cg),
  // hi(rho) on 2^-kGridT.  Exactness in units of U (|hi(alpha)|, |hi(rho)| <= 1.0004):
  // hi(Y) sums on U 2^-21 with partial sums <= 1.5 U; |Y| <= 1.42 U, so hi(X) = hi(Y_0) +
  // hi(rho) hi(Y_1) sums on U 2^-21 stay below 2.84 U; |X| <= 2.84 U, so hi(E') =
  // hi(X[.][0]) + hi(X[.][1]) hi(conj b) sums on U 2^-21 stay below 5.7 U (< 2^24 units).
  // Every kRenormEvery sites (all threads at once) an exact power-of-two rescale, counted
  // in L, brings e back to 0; a guard rescales at once if e leaves +-96 in between.
  static constexpr int kRenormEvery = 8;
  using Rec = Record<4, QSVM_FP32_SPLIT>;
  float2 Eh[2][2][2], El[2][2][2];
  float Cg;  // 1.5 * 2^(e + 14): adding and subtracting it rounds to the grid U 2^-10
  int eE;    // e of the current environment
  int L;

  __device__ __forceinline__ void init() {
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int r = 0; r < 2; ++r) Eh[c][q][r] = El[c][q][r] = make_float2(0.f, 0.f);
    Eh[0][0][0].x = 1.f;
    eE = 1;  // E = e_0 e_0^T: largest component 1
    Cg = grid_const(eE);
    L = 2;  // every site() counts -2 for the factors 1/2 of a and b; the virtual site has none
  }

  // split forms of value v of a record (a-form array: (V, iV); b-form array: (conj V, i conj V))
  static __device__ __forceinline__ SplitForm form(uint32_t rec, int v) {
    SplitForm F;
    const float4 qh = *reinterpret_cast<const float4*>(sptr(rec + Rec::off(v, 0)));
    const float4 ql = *reinterpret_cast<const float4*>(sptr(rec + Rec::off(v, 1)));
    F.h = make_float2(qh.x, qh.y);
    F.ih = make_float2(qh.z, qh.w);
    F.l = make_float2(ql.x, ql.y);
    F.il = make_float2(ql.z, ql.w);
    return F;
  }
  // (hh, ll) += w V for a split w (hi, lo, full) and a split form of V
  static __device__ __forceinline__ void smac(float2& hh, float2& ll, float2 wh, float2 wl, float2 wf,
                                              const SplitForm& V) {
    hh = fma2(bc(wh.x), V.h, hh);
    hh = fma2(bc(wh.y), V.ih, hh);
    ll = fma2(bc(wl.x), V.h, ll);
    ll = fma2(bc(wl.y), V.ih, ll);
    ll = fma2(bc(wf.x), V.l, ll);
    ll = fma2(bc(wf.y), V.il, ll);
  }
  // 1.5 * 2^(e + 14) for the frexp exponent e (|e| <= 32 here)
  static __device__ __forceinline__ float grid_const(int e) {
    return __int_as_float(((127 + 14 + e) << 23) | 0x400000);
  }
  // re-split onto the grid of the rounding constant C
  static __device__ __forceinline__ void ssplit(float2 hh, float2 ll, float C, float2& xh, float2& xl, float2& xf) {
    const float2 v = add2(hh, ll);
    xh = add2(add2(v, bc(C)), bc(-C));
    xl = add2(fma2(xh, make_float2(-1.f, -1.f), hh), ll);  // (hh - xh) is exact
    xf = v;
  }

  __device__ __forceinline__ void site(uint32_t ra, uint32_t rb) {
    // Y_c = a^T E_c for both blocks (Y_0 unsplit, Y_1 split onto 2^-GG)
    float2 Y0h[2][2], Y0l[2][2], Y1h[2][2], Y1l[2][2], Y1f[2][2];
    {
      const SplitForm A0 = form(ra, 0), A1 = form(ra, 1);
#pragma unroll
      for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int p = 0; p < 2; ++p) {
          float2 hh = Eh[0][0][r], ll = El[0][0][r];
          smac(hh, ll, Eh[0][1][r], El[0][1][r], add2(Eh[0][1][r], El[0][1][r]), p ? A1 : A0);
          Y0h[p][r] = hh;
          Y0l[p][r] = ll;
          hh = Eh[1][0][r];
          ll = El[1][0][r];
          smac(hh, ll, Eh[1][1][r], El[1][1][r], add2(Eh[1][1][r], El[1][1][r]), p ? A1 : A0);
          ssplit(hh, ll, Cg, Y1h[p][r], Y1l[p][r], Y1f[p][r]);
        }
    }
    const SplitForm B0 = form(rb, 0), B1 = form(rb, 1);
    float2 Nh[2][2][2], Nl[2][2][2];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      // X_s = Y_0 + rho_s Y_1, then E'_s = X_s conj(b); rho_s is formed here, so that
      // only one of the two is live at a time (0.7 % faster than forming both first)
      SplitForm R;
      split_rho(ra + Rec::off(s, 0), ra + Rec::off(s, 1), rb + Rec::off(s, 0), rb + Rec::off(s, 1), R.h, R.ih, R.l,
                R.il);
      float2 Xh[2][2], Xl[2][2], Xf[2][2];
#pragma unroll
      for (int p = 0; p < 2; ++p)
#pragma unroll
        for (int r = 0; r < 2; ++r) {
          float2 hh = Y0h[p][r], ll = Y0l[p][r];
          smac(hh, ll, Y1h[p][r], Y1l[p][r], Y1f[p][r], R);
          if (r) {
            ssplit(hh, ll, Cg, Xh[p][r], Xl[p][r], Xf[p][r]);
          } else {  // seeds E'_s[p][.]
            Xh[p][r] = hh;
            Xl[p][r] = ll;
          }
        }
#pragma unroll
      for (int p = 0; p < 2; ++p)
#pragma unroll
        for (int pp = 0; pp < 2; ++pp) {
          float2 hh = Xh[p][0], ll = Xl[p][0];
          smac(hh, ll, Xh[p][1], Xl[p][1], Xf[p][1], pp ? B1 : B0);
          Nh[s][p][pp] = hh;
          Nl[s][p][pp] = ll;
        }
    }
    // the new environment: its exponent sets this site's grid; an exact rescale keeps e
    // within +-32; the signs (-1)^{p+pp} of S E_1 S are applied; re-split onto U 2^-10
    const float2 m1 = make_float2(-1.f, -1.f);
    float2 V[2][2][2];
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int p = 0; p < 2; ++p)
#pragma unroll
        for (int r = 0; r < 2; ++r) V[s][p][r] = add2(Nh[s][p][r], Nl[s][p][r]);
    float m = max_abs<8>(reinterpret_cast<const float2(&)[8]>(V));
    int e = (m > 0.f && isfinite(m)) ? exp_of(m) : 0;
    if (e > 96 || e < -96) {  // rare guard between the periodic rescales
      const float2 sc = bc(pow2f(-e));
#pragma unroll
      for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int p = 0; p < 2; ++p)
#pragma unroll
          for (int r = 0; r < 2; ++r) {
            Nh[s][p][r] = mul2(Nh[s][p][r], sc);
            Nl[s][p][r] = mul2(Nl[s][p][r], sc);
            V[s][p][r] = mul2(V[s][p][r], sc);
          }
      L += e;
      m = max_abs<8>(reinterpret_cast<const float2(&)[8]>(V));
      e = (m > 0.f && isfinite(m)) ? exp_of(m) : 0;
    }
    eE = e;
    Cg = grid_const(e);
    const float2 cp = bc(Cg), cm = bc(-Cg);
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int p = 0; p < 2; ++p)
#pragma unroll
        for (int r = 0; r < 2; ++r) {
          const float2 h = add2(add2(V[s][p][r], cp), cm);
          const float2 l = add2(fma2(h, m1, Nh[s][p][r]), Nl[s][p][r]);  // (Nh - h) is exact
          if (s == 1 && ((p + r) & 1)) {
            Eh[s][p][r] = mul2(h, m1);
            El[s][p][r] = mul2(l, m1);
          } else {
            Eh[s][p][r] = h;
            El[s][p][r] = l;
          }
        }
    L -= 2;
  }

  // periodic rescale by 2^-e (exact; every thread of the warp at the same site)
  __device__ __forceinline__ void renorm() {
    const float2 sc = bc(pow2f(-eE));
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int p = 0; p < 2; ++p)
#pragma unroll
        for (int r = 0; r < 2; ++r) {
          Eh[s][p][r] = mul2(Eh[s][p][r], sc);
          El[s][p][r] = mul2(El[s][p][r], sc);
        }
    L += eE;
    eE = 0;
    Cg = grid_const(0);
  }

  // after the virtual site the amplitude is entry (0, 0) of block 0 (up to a phase)
  __device__ __forceinline__ void amplitude(double& re, double& im) const {
    re = __dadd_rn((double)Eh[0][0][0].x, (double)El[0][0][0].x);
    im = __dadd_rn((double)Eh[0][0][0].y, (double)El[0][0][0].y);
  }
};

// ------------------------------------------------------- tile kernel ------
// Device status word of this translation unit (QSVM_OK or QSVM_ERR_TIMEOUT).
__device__ int32_t g_pair_status;

// Split FP32 at chi = 8 with four threads per pair.  One thread cannot hold a
// pair's split environment (2 blocks x 16 entries, hi and lo) next to its
// working set, so the quad shares it: each thread keeps one column of both blocks
// in registers, and the entries change hands twice per site through a 512-byte
// buffer per pair (warp barriers separate its writes and reads).  The quad agrees
// on the power-of-two rescale through two xor-shuffles.  The records are the
// gauged ones of reps = 2 (the same alpha and beta; see QuadEngine below).
template <int PREC>
struct QuadEngine;

template <>
struct QuadEngine<QSVM_FP32_SPLIT> {
  // Gauged form at reps = 3: both blocks of a site are the signed Kronecker square
  // a[q][p] = (-1)^{q1 q2} M[q1][p1] M[q2][p2] of M = [[1, 1], [alpha, beta]] (q = q1 + 2 q2,
  // p = p1 + 2 p2) and block c = 1 adds r'_s S with S = diag(1, 1, -1, -1) (r'_0 = alpha,
  // r'_1 = beta), so with the row signs T = diag(1, 1, 1, -1) folded into the stored
  // environment, Ev_c = T S^c E_c S^c T, a site is
  //   Y_c = (M_i x M_i)^T Ev_c,  X_s = Y_0 + rho_s Y_1,  E'_s = X_s conj(M_j x M_j),
  // each Kronecker product applied as two 2 x 2 stages (Z over q1, Y over q2; W over r1,
  // E' over r2): 40 complex MACs per thread and 160 per pair per site.  Thread t of the
  // quad owns column r = t of both blocks for the row stages and the mix, and row p = t of
  // both X_s for the column stages; X and E' change hands through the pair's shared buffer.
  // Grids: E's components below 1/4 after renormalisation, hi(E) on 2^-GE (2^-11);
  // hi(Z) of the multiplied rows and hi(Y_1) on 2^-10 (Z and Y partial sums on 2^-22,
  // below 0.75 and 1.5; X = Y_0 + rho Y_1 on 2^-22, below 2.9); X fully re-split onto 2^-9
  // (it changes hands); W's multiplied entries re-split onto 2^-9, its other entries seed
  // E' unsplit (|W| <= 5.7 on 2^-20); E' below 11.4 on 2^-20: every partial sum stays
  // below 2^24 units.
  static constexpr int CHI = 8, H = 4;
  static constexpr int GE = 11, GZ = 10, GY = 10, GX = 9, GW = 9;
  static constexpr int kRenormEvery = 1;
  using Rec = Record<CHI, QSVM_FP32_SPLIT>;
  float* ebuf;     // this pair's 32-entry exchange buffer (see entry())
  int t, pi;       // thread of the quad, parity of the pair
  unsigned mask;   // the warp's active mask (all 32 lanes run the site loop together)
  float2 Eh[2][H], El[2][H];  // column t of both blocks of the (sign-folded) environment
  int L;

  __device__ __forceinline__ void init(float* pair_buf, int quarter) {
    ebuf = pair_buf;
    t = quarter;
    pi = (int)((threadIdx.x >> 2) & 1);
    mask = 0xffffffffu;
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int q = 0; q < H; ++q) Eh[c][q] = El[c][q] = make_float2(0.f, 0.f);
    if (t == 0) Eh[0][0].x = 1.f;  // E_0 = e_0 e_0^T
    L = 3;  // every site() counts -3 for the factors 2^{-3/2} of a and b; the virtual site has none
  }

  // Entry (a, row, col) of the exchange buffer, 16 bytes.  The eight threads of a
  // quarter-warp (two pairs) write (a, row, t) and read (a, t, col) for fixed (a, row) or
  // (a, col); flipping the row's low bit and the column's high bit with the pair's parity
  // and the column's low bit with the row's high bit puts them in eight different 16-byte
  // bank groups in both patterns.
  __device__ __forceinline__ float4* entry(int a, int row, int col) const {
    return reinterpret_cast<float4*>(ebuf) + (a * 16 + 4 * (row ^ pi) + (col ^ (row >> 1) ^ (2 * pi)));
  }

  static __device__ __forceinline__ SplitForm form(uint32_t rec, int v) {
    SplitForm F;
    const float4 qh = *reinterpret_cast<const float4*>(sptr(rec + Rec::off(v, 0)));
    const float4 ql = *reinterpret_cast<const float4*>(sptr(rec + Rec::off(v, 1)));
    F.h = make_float2(qh.x, qh.y);
    F.ih = make_float2(qh.z, qh.w);
    F.l = make_float2(ql.x, ql.y);
    F.il = make_float2(ql.z, ql.w);
    return F;
  }
  // (hh, ll) += w V for a split w (hi, lo, full) and a split form of V
  static __device__ __forceinline__ void smac(float2& hh, float2& ll, float2 wh, float2 wl, float2 wf,
                                              const SplitForm& V) {
    hh = fma2(bc(wh.x), V.h, hh);
    hh = fma2(bc(wh.y), V.ih, hh);
    ll = fma2(bc(wl.x), V.h, ll);
    ll = fma2(bc(wl.y), V.ih, ll);
    ll = fma2(bc(wf.x), V.l, ll);
    ll = fma2(bc(wf.y), V.il, ll);
  }
  template <int GS>
  static __device__ __forceinline__ void ssplit(float2 hh, float2 ll, float2& xh, float2& xl, float2& xf) {
    const float2 v = add2(hh, ll);
    xh = grid_round2<GS>(v);
    xl = add2(fma2(xh, make_float2(-1.f, -1.f), hh), ll);  // (hh - xh) is exact
    xf = v;
  }

  __device__ __forceinline__ void site(uint32_t ra, uint32_t rb) {
    const float2 m1 = make_float2(-1.f, -1.f);
    // ---- rows of column t: Y_c = (M_i x M_i)^T Ev_c, X_s = Y_0 + rho_s Y_1 ----
    float2 Xh[2][H], Xl[2][H];
    {
      const SplitForm A[2] = {form(ra, 0), form(ra, 1)};
      float2 Y0h[H], Y0l[H], Y1h[H], Y1l[H], Y1f[H];
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        // Z[p1 + 2 q2] = Ev[2 q2] + M[p1] Ev[1 + 2 q2]: rows with q2 = 1 re-split (they are multiplied next)
        float2 Zh[H], Zl[H], Zf[H];
#pragma unroll
        for (int q2 = 0; q2 < 2; ++q2) {
          const float2 wh = Eh[c][1 + 2 * q2], wl = El[c][1 + 2 * q2], wf = add2(wh, wl);
#pragma unroll
          for (int p1 = 0; p1 < 2; ++p1) {
            float2 hh = Eh[c][2 * q2], ll = El[c][2 * q2];
            smac(hh, ll, wh, wl, wf, A[p1]);
            if (q2) {
              ssplit<GZ>(hh, ll, Zh[p1 + 2], Zl[p1 + 2], Zf[p1 + 2]);
            } else {
              Zh[p1] = hh;
              Zl[p1] = ll;
            }
          }
        }
        // Y[p1 + 2 p2] = Z[p1] + M[p2] Z[p1 + 2]: Y_1 re-split (multiplied by rho next)
#pragma unroll
        for (int p2 = 0; p2 < 2; ++p2)
#pragma unroll
          for (int p1 = 0; p1 < 2; ++p1) {
            float2 hh = Zh[p1], ll = Zl[p1];
            smac(hh, ll, Zh[p1 + 2], Zl[p1 + 2], Zf[p1 + 2], A[p2]);
            if (c) {
              ssplit<GY>(hh, ll, Y1h[p1 + 2 * p2], Y1l[p1 + 2 * p2], Y1f[p1 + 2 * p2]);
            } else {
              Y0h[p1 + 2 * p2] = hh;
              Y0l[p1 + 2 * p2] = ll;
            }
          }
      }
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        SplitForm R;  // rho_s, formed where it is used (one live at a time)
        split_rho(ra + Rec::off(s, 0), ra + Rec::off(s, 1), rb + Rec::off(s, 0), rb + Rec::off(s, 1), R.h, R.ih, R.l,
                  R.il);
#pragma unroll
        for (int p = 0; p < H; ++p) {
          float2 hh = Y0h[p], ll = Y0l[p], xf;
          smac(hh, ll, Y1h[p], Y1l[p], Y1f[p], R);
          ssplit<GX>(hh, ll, Xh[s][p], Xl[s][p], xf);
        }
      }
    }
    // ---- X changes hands: thread t takes row p = t of both X_s ----
    __syncwarp(mask);  // every thread has read the previous site's environment entries
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int p = 0; p < H; ++p) *entry(s, p, t) = make_float4(Xh[s][p].x, Xh[s][p].y, Xl[s][p].x, Xl[s][p].y);
    __syncwarp(mask);
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int r = 0; r < H; ++r) {
        const float4 v = *entry(s, t, r);
        Xh[s][r] = make_float2(v.x, v.y);
        Xl[s][r] = make_float2(v.z, v.w);
      }
    // ---- columns of row t: E'_s = X_s conj(M_j x M_j) ----
    float2 Nh[2][H], Nl[2][H];
    {
      const SplitForm B[2] = {form(rb, 0), form(rb, 1)};
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        // W[pp1 + 2 r2] = X[2 r2] + conj(M[pp1]) X[1 + 2 r2]: entries with r2 = 1 re-split
        // (they are multiplied next), the others seed E'
        float2 Wh[H], Wl[H], Wf[H];
#pragma unroll
        for (int r2 = 0; r2 < 2; ++r2) {
          const float2 wh = Xh[s][1 + 2 * r2], wl = Xl[s][1 + 2 * r2], wf = add2(wh, wl);
#pragma unroll
          for (int pp1 = 0; pp1 < 2; ++pp1) {
            float2 hh = Xh[s][2 * r2], ll = Xl[s][2 * r2];
            smac(hh, ll, wh, wl, wf, B[pp1]);
            if (r2) {
              ssplit<GW>(hh, ll, Wh[pp1 + 2], Wl[pp1 + 2], Wf[pp1 + 2]);
            } else {
              Wh[pp1] = hh;
              Wl[pp1] = ll;
            }
          }
        }
        // E'[pp1 + 2 pp2] = W[pp1] + conj(M[pp2]) W[pp1 + 2]
#pragma unroll
        for (int pp2 = 0; pp2 < 2; ++pp2)
#pragma unroll
          for (int pp1 = 0; pp1 < 2; ++pp1) {
            float2 hh = Wh[pp1], ll = Wl[pp1];
            smac(hh, ll, Wh[pp1 + 2], Wl[pp1 + 2], Wf[pp1 + 2], B[pp2]);
            Nh[s][pp1 + 2 * pp2] = hh;
            Nl[s][pp1 + 2 * pp2] = ll;
          }
      }
    }
    // ---- quad-wide renormalisation to components below 1/4, signs T S^s . S^s T ----
    float2 V[2][H];
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int pp = 0; pp < H; ++pp) V[s][pp] = add2(Nh[s][pp], Nl[s][pp]);
    float m = max_abs<2 * H>(reinterpret_cast<const float2(&)[2 * H]>(V));
    m = fmaxf(m, __shfl_xor_sync(mask, m, 1));
    m = fmaxf(m, __shfl_xor_sync(mask, m, 2));
    int e = 0;
    if (m > 0.f && isfinite(m)) {
      e = exp_of(m);
      if (e < -120) {  // collapse to near zero: scale up in two exact steps
        const float2 up = bc(pow2f(100));
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
          for (int pp = 0; pp < H; ++pp) {
            Nh[s][pp] = mul2(Nh[s][pp], up);
            Nl[s][pp] = mul2(Nl[s][pp], up);
            V[s][pp] = mul2(V[s][pp], up);
          }
        L -= 100;
        e += 100;
      }
    }
    const float sc = pow2f(-(e + 2));
    const int tt = (t == 3), ts = (t >> 1);  // T and S sign bits of row t
    __syncwarp(mask);  // every thread has read its row of X
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int pp = 0; pp < H; ++pp) {
        const int neg = (tt ^ (pp == 3) ^ (s & (ts ^ (pp >> 1)))) & 1;
        const float2 scs = bc(neg ? -sc : sc);
        const float2 f = mul2(V[s][pp], scs);
        const float2 hv = grid_round2<GE>(f);
        const float2 lv = fma2(Nl[s][pp], scs, fma2(hv, m1, mul2(Nh[s][pp], scs)));
        *entry(s, t, pp) = make_float4(hv.x, hv.y, lv.x, lv.y);
      }
    __syncwarp(mask);
    // ---- the new environment changes hands: thread t takes column t ----
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int q = 0; q < H; ++q) {
        const float4 v = *entry(c, q, t);
        Eh[c][q] = make_float2(v.x, v.y);
        El[c][q] = make_float2(v.z, v.w);
      }
    L += e + 2 - 3;
  }

  __device__ __forceinline__ void renorm() {}

  // after the virtual site the amplitude is entry (0, 0) of block 0 (up to a phase); the
  // writer is thread 0 of the quad, which holds column 0
  __device__ __forceinline__ void amplitude(double& re, double& im) const {
    re = __dadd_rn((double)Eh[0][0].x, (double)El[0][0].x);
    im = __dadd_rn((double)Eh[0][0].y, (double)El[0][0].y);
  }
};

constexpr int kMaxStages = 4;
constexpr int kCtlBytes = 128;

// Tile geometry.  The Gram and cross kernels are cut into tiles of tile_side x
// tile_side pairs (16 x 16; 8 x 8 for split FP32 at chi = 8, which runs four threads
// per pair, QuadEngine); tile indices, partitions and tile lists use this side.  A
// CTA contracts either a whole tile or, with a sub-tile configuration, one of its
// 2 x 2 quarters (8 x 8 or 4 x 4 pairs), so a launch runs 4 CTAs per tile; the
// pipeline configuration picks which (an autotuner knob).
__host__ __device__ constexpr int threads_per_pair(int chi, int prec) {
  return (chi >= 8 && prec == QSVM_FP32_SPLIT) ? 4 : 1;
}
__host__ __device__ constexpr int tile_side(int chi, int prec) { return threads_per_pair(chi, prec) == 4 ? 8 : 16; }
// threads of a CTA that contracts a ti x ti block of pairs with tpp threads per pair
__host__ __device__ constexpr int cta_threads(int ti, int tpp) { return ti * ti * tpp; }
__host__ __device__ constexpr int out_bytes(int ti) { return ti * (ti + 1) * 16; }
// shared environment buffer of the four-thread layout: 32 entries x 16 B per pair,
// padded to 36 entries (a stride of 4 mod 8 sixteen-byte bank groups)
constexpr int kQuadPairFloats = 32 * 4;  // the four-thread engine's exchange buffer per pair
__host__ __device__ constexpr int ebuf_bytes(int chi, int prec, int ti) {
  return threads_per_pair(chi, prec) == 4 ? ti * ti * kQuadPairFloats * 4 : 0;
}

// CTAs per SM the register budget is set for; a sub-tile CTA (SUB = 2) has a
// quarter of the threads, so four times as many keep the same warps resident
template <int CHI, int PREC, int SUB>
__host__ __device__ constexpr int min_blocks_per_sm() {
  return SUB * SUB * ((threads_per_pair(CHI, PREC) == 4) ? 2 : (CHI >= 8) ? 1 : ((PREC == QSVM_FP32) ? 3 : 2));
}
template <int CHI, int PREC, int SUB>
__host__ __device__ constexpr int kernel_threads() {
  return cta_threads(tile_side(CHI, PREC) / SUB, threads_per_pair(CHI, PREC));
}

// Shared-memory control block at the end of the dynamic allocation.
struct TileCtl {
  uint64_t bars[kMaxStages];  // one "full" mbarrier per stage
  int done[kMaxStages];       // warps finished with the stage's current chunk
  int abort_flag;             // a wait timed out somewhere in the CTA
  int issued;                 // chunks issued (global count)
  long long next_tile;        // persistent kernel: tile fetched for the CTA
};
static_assert(sizeof(TileCtl) <= kCtlBytes, "control block");

// Dynamic shared memory: stages | output tile (K, logK) | control block | environment buffer (4-thread layout)
__host__ __device__ inline int pipe_smem_bytes(const PipeCfg& pc, int chi, int prec) {
  return pc.stages * pc.stage_bytes + out_bytes(pc.tile) + kCtlBytes + ebuf_bytes(chi, prec, pc.tile);
}

// What one tile needs to know.
struct TileWork {
  const uint8_t* mpsA;
  const uint8_t* mpsB;
  int64_t nA, nB;
  int64_t ti, tj;
  int n;
  int symmetric;
  double* K;
  int64_t ldk;
  double* logK;
  int64_t ldl;
};

// Contract one TI x TI tile of pairs.  Site records stream through a ring of
// pc.stages shared-memory stages of pc.S sites each.  Stage refill needs no
// CTA-wide barrier: each warp, after computing a chunk, counts itself out on the
// stage's counter, and the warp that completes the count issues the bulk copies
// of the chunk pc.stages ahead into that stage; warps only wait for data.
// gchunk is the CTA's running chunk count (stage and mbarrier parity continue
// across the tiles a persistent CTA processes).  Returns false after a timeout.
template <int CHI, int PREC, int TPP>
struct EngineFor {
  using type = Engine<CHI, PREC>;
};
template <int CHI, int PREC>
struct EngineFor<CHI, PREC, 4> {
  using type = QuadEngine<PREC>;
};

// TI is the side of the block of pairs this CTA contracts (a tile or a sub-tile);
// w.ti and w.tj count in units of TI.
template <int CHI, int PREC, int TI>
__device__ __forceinline__ bool run_tile(const TileWork& w, const PipeCfg& pc, uint8_t* smem, TileCtl* ctl,
                                         int& gchunk) {
  using Rec = Record<CHI, PREC>;
  constexpr int TPP = threads_per_pair(CHI, PREC);
  constexpr int kWarps = cta_threads(TI, TPP) / 32;
  using Eng = typename EngineFor<CHI, PREC, TPP>::type;
  const int S = pc.S, NST = pc.stages, SLOT = pc.slot_bytes, STAGE = pc.stage_bytes;
  double* outK = reinterpret_cast<double*>(smem + NST * STAGE);
  double* outL = outK + TI * (TI + 1);

  const int64_t i0 = w.ti * TI, j0 = w.tj * TI;
  const int ni = (int)((w.nA - i0) < TI ? (w.nA - i0) : TI);
  const int nj = (int)((w.nB - j0) < TI ? (w.nB - j0) : TI);
  const int n = record_sites(w.n, CHI, PREC);  // records per point (sites, plus a virtual one)
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int pair = tid / TPP, quarter = tid % TPP;
  const int ty = pair / TI, tx = pair % TI;
  const bool diag_tile = w.symmetric && w.ti == w.tj;
  const bool valid = ty < ni && tx < nj && (!diag_tile || ty <= tx);
  const int slotA = min(ty, ni - 1);
  const int slotB = TI + min(tx, nj - 1);
  const int nchunks = (n + S - 1) / S;
  const int g0 = gchunk;

  // Issue chunk ch into its stage, by one whole warp: lane 0 posts the expected
  // bytes on the stage's mbarrier, then lane l < ni copies row point l and lane
  // ni + l < ni + nj column point l (ni + nj <= 2 TI <= 32).
  auto issue = [&](int ch) {
    const int g = g0 + ch;
    const int st = g % NST;
    const int k0 = ch * S;
    const int ns = min(S, n - k0);
    const uint32_t bytes = (uint32_t)(ns * Rec::kBytes);
    if (lane == 0) mbar_arrive_expect_tx(&ctl->bars[st], bytes * (uint32_t)(ni + nj));
    __syncwarp();
    uint8_t* base = smem + st * STAGE;
    if (lane < ni) {
      bulk_g2s(base + lane * SLOT, w.mpsA + ((i0 + lane) * (int64_t)n + k0) * Rec::kBytes, bytes, &ctl->bars[st]);
    } else if (lane < ni + nj) {
      const int p = lane - ni;
      bulk_g2s(base + (TI + p) * SLOT, w.mpsB + ((j0 + p) * (int64_t)n + k0) * Rec::kBytes, bytes, &ctl->bars[st]);
    }
    if (lane == 0) ctl->issued = g + 1;
  };
  static_assert(2 * TI <= 32, "one lane per point of a tile");

  if (tid < 32)
    for (int ch = 0; ch < min(NST, nchunks); ++ch) issue(ch);
  __syncthreads();

  Eng eng;
  if constexpr (TPP == 4) {
    float* ebuf = reinterpret_cast<float*>(smem + NST * STAGE + out_bytes(TI) + kCtlBytes) + pair * kQuadPairFloats;
    eng.init(ebuf, quarter);
  } else {
    eng.init();
  }
  for (int ch = 0; ch < nchunks; ++ch) {
    const int g = g0 + ch;
    const int st = g % NST;
    const uint32_t parity = (uint32_t)((g / NST) & 1);
    // bounded wait for the chunk; give up early if another warp already timed out
    bool ok = mbar_try_wait(&ctl->bars[st], parity);
    if (!ok) {
      const uint64_t t0 = global_ns();
      while (!(ok = mbar_try_wait(&ctl->bars[st], parity))) {
        if (*(volatile int*)&ctl->abort_flag || global_ns() - t0 > kWaitLimitNs) break;
      }
    }
    ok = __all_sync(0xffffffffu, ok);  // the warp acts on one outcome
    if (!ok) {
      if (lane == 0) *(volatile int*)&ctl->abort_flag = 1;
      break;
    }
    const uint32_t base = smem_u32(smem) + st * STAGE;
    const int k0 = ch * S;
    const int ns = min(S, n - k0);
    // the four-thread layout synchronises the warp inside site(), so every pair of
    // such a tile computes (on clamped points if it is outside the tile) and only
    // valid pairs write results
    if (valid || TPP > 1) {
      const uint32_t pa = base + slotA * SLOT;
      const uint32_t pb = base + slotB * SLOT;
      if constexpr (PREC == QSVM_FP32_SPLIT && TPP == 1) {
        // two sites per iteration let the compiler start a site's shared loads
        // during the previous site's renormalisation (within the register budget)
#pragma unroll 2
        for (int s = 0; s < ns; ++s) {
          eng.site(pa + s * Rec::kBytes, pb + s * Rec::kBytes);
          if (Eng::kRenormEvery > 1 && ((k0 + s + 1) % Eng::kRenormEvery) == 0) eng.renorm();
        }
      } else {
#pragma unroll 1
        for (int s = 0; s < ns; ++s) {
          eng.site(pa + s * Rec::kBytes, pb + s * Rec::kBytes);
          if (Eng::kRenormEvery > 1 && ((k0 + s + 1) % Eng::kRenormEvery) == 0) eng.renorm();
        }
      }
    }
    __syncwarp();
    // all shared-memory reads of this warp for the stage are complete (their
    // values were consumed above); count the warp out and, if last, refill
    int last = 0;
    if (lane == 0) {
      __threadfence_block();
      last = atomicAdd(&ctl->done[st], 1) == kWarps - 1;
      if (last) ctl->done[st] = 0;
    }
    last = __shfl_sync(0xffffffffu, last, 0);
    if (last && ch + NST < nchunks) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(ch + NST);
    }
  }
  __syncthreads();
  gchunk = g0 + nchunks;

  if (ctl->abort_flag) {
    // A copy never completed: record it, wait (bounded) for the copies this CTA
    // may still have in flight, and stop without writing results.
    if (tid == 0) {
      atomicCAS(&g_pair_status, 0, (int32_t)QSVM_ERR_TIMEOUT);
      const int last = ctl->issued;
      for (int g = max(0, last - NST); g < last; ++g)
        mbar_wait_bounded(&ctl->bars[g % NST], (uint32_t)((g / NST) & 1), kDrainLimitNs);
    }
    return false;
  }

  double kval = 0.0, lval = -INFINITY;
  const bool writer = valid && quarter == 0;
  if (writer) {
    if (Eng::kRenormEvery > 1) eng.renorm();
    double re, im;
    eng.amplitude(re, im);
    // explicit roundings, so every kernel that runs this epilogue gives the same bits
    const double a2 = __fma_rn(re, re, __dmul_rn(im, im));
    if (a2 > 0.0) {
      kval = ldexp(a2, 2 * eng.L);
      lval = __fma_rn((double)(2 * eng.L), 0.69314718055994530942, log(a2));
    }
    w.K[(i0 + ty) * w.ldk + (j0 + tx)] = kval;
    if (w.logK) w.logK[(i0 + ty) * w.ldl + (j0 + tx)] = lval;
  }
  if (w.symmetric) {
    // mirror K[j][i] = K[i][j] bit-exactly, through shared memory so that the
    // transposed rows are written contiguously
    if (quarter == 0) {
      outK[ty * (TI + 1) + tx] = kval;
      outL[ty * (TI + 1) + tx] = lval;
    }
    __syncthreads();
    // this thread writes row j0+ty, column i0+tx: the value of pair (i0+tx, j0+ty)
    const bool src = quarter == 0 && tx < ni && ty < nj && (!diag_tile || tx < ty);
    if (src) {
      w.K[(j0 + ty) * w.ldk + (i0 + tx)] = outK[tx * (TI + 1) + ty];
      if (w.logK) w.logK[(j0 + ty) * w.ldl + (i0 + tx)] = outL[tx * (TI + 1) + ty];
    }
    __syncthreads();  // outK is reused by the next tile of a persistent CTA
  }
  return true;
}

// the control block of a CTA whose block of pairs has side TI (== pc.tile)
template <int TI>
__device__ __forceinline__ TileCtl* tile_ctl(uint8_t* smem, const PipeCfg& pc) {
  return reinterpret_cast<TileCtl*>(smem + pc.stages * pc.stage_bytes + out_bytes(TI));
}

__device__ __forceinline__ void tile_ctl_init(TileCtl* ctl, const PipeCfg& pc) {
  if (threadIdx.x == 0) {
    for (int s = 0; s < pc.stages; ++s) {
      mbar_init(&ctl->bars[s], 1);
      ctl->done[s] = 0;
    }
    ctl->abort_flag = 0;
    ctl->issued = 0;
    fence_mbar_init();
  }
  __syncthreads();
}

// One CTA per tile of a launch (grid = number of tiles in [tile_begin, ...)), or,
// with SUB = 2, one CTA per quarter of a tile (grid = 4 x tiles): CTA 4t + 2qi + qj
// takes quarter (qi, qj) of tile t.  In a diagonal tile of a Gram the quarter
// (1, 0) lies below the diagonal (its entries are the mirror of quarter (0, 1)),
// and quarters beyond a ragged last tile row or column hold no pairs: such CTAs
// return at once.
template <int CHI, int PREC, int SUB>
__global__ void __launch_bounds__(kernel_threads<CHI, PREC, SUB>(), (min_blocks_per_sm<CHI, PREC, SUB>()))
    pair_tile_kernel(TileArgs args, PipeCfg pc) {
  constexpr int TI = tile_side(CHI, PREC) / SUB;
  uint8_t* smem = qsvm_dyn_smem;
  TileCtl* ctl = tile_ctl<TI>(smem, pc);
  TileWork w;
  if constexpr (SUB > 1) {
    const int64_t b = args.tile_begin + blockIdx.x / (SUB * SUB);
    const int qi = (int)(blockIdx.x % (SUB * SUB)) / SUB, qj = (int)(blockIdx.x % (SUB * SUB)) % SUB;
    if (args.symmetric) sym_tile_decode(b, args.tiles_j, w.ti, w.tj);
    else rect_tile_decode(b, args.tiles_i, args.tiles_j, w.ti, w.tj);
    if (args.symmetric && w.ti == w.tj && qi > qj) return;
    w.ti = w.ti * SUB + qi;
    w.tj = w.tj * SUB + qj;
    if (w.ti * TI >= args.nA || w.tj * TI >= args.nB) return;
    tile_ctl_init(ctl, pc);
  } else {
    tile_ctl_init(ctl, pc);
    const int64_t b = args.tile_begin + blockIdx.x;
    if (args.symmetric) sym_tile_decode(b, args.tiles_j, w.ti, w.tj);
    else rect_tile_decode(b, args.tiles_i, args.tiles_j, w.ti, w.tj);
  }
  w.mpsA = args.mpsA;
  w.mpsB = args.mpsB;
  w.nA = args.nA;
  w.nB = args.nB;
  w.n = args.n;
  w.symmetric = args.symmetric;
  w.K = args.K;
  w.ldk = args.ldk;
  w.logK = args.logK;
  w.ldl = args.ldl;
  int gchunk = 0;
  run_tile<CHI, PREC, TI>(w, pc, smem, ctl, gchunk);
}

// Persistent kernel over a queue of Gram tiles from many jobs: every CTA pulls
// the next tile index from a device counter until the queue is empty.  Jobs are
// ordered heaviest first by the host; tile t belongs to the job j with
// prefix[j] <= t < prefix[j + 1].  Always whole tiles (pc.tile == tile_side).
template <int CHI, int PREC>
__global__ void __launch_bounds__(kernel_threads<CHI, PREC, 1>(), (min_blocks_per_sm<CHI, PREC, 1>()))
    pair_persistent_kernel(BatchArgs args, PipeCfg pc) {
  uint8_t* smem = qsvm_dyn_smem;
  TileCtl* ctl = tile_ctl<tile_side(CHI, PREC)>(smem, pc);
  tile_ctl_init(ctl, pc);
  int gchunk = 0;
  while (true) {
    if (threadIdx.x == 0) ctl->next_tile = (long long)atomicAdd(args.counter, 1ull);
    __syncthreads();
    const int64_t t = (int64_t)ctl->next_tile;
    __syncthreads();  // next_tile is rewritten on the next iteration
    if (t >= args.total_tiles) break;
    int lo = 0, hi = args.n_jobs - 1;  // last job whose prefix <= t
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (args.prefix[mid] <= t) lo = mid;
      else hi = mid - 1;
    }
    const DevJob& J = args.jobs[lo];
    TileWork w;
    sym_tile_decode(t - args.prefix[lo], J.tiles, w.ti, w.tj);
    w.mpsA = J.mps;
    w.mpsB = J.mps + (Record<CHI, PREC>::kForms == 2
                          ? J.n_points * (int64_t)record_sites(J.n_qubits, CHI, PREC) * Record<CHI, PREC>::kBytes
                          : 0);
    w.nA = w.nB = J.n_points;
    w.n = J.n_qubits;
    w.symmetric = 1;
    w.K = J.K;
    w.ldk = J.ldk;
    w.logK = J.logK;
    w.ldl = J.ldl;
    if (!run_tile<CHI, PREC, tile_side(CHI, PREC)>(w, pc, smem, ctl, gchunk)) break;
  }
}

}  // namespace qsvm
