// qsvm_common.cuh -- device-side helpers shared by the libqsvm kernels.
//
// Site-record layouts (see include/qsvm.h): reps = 1, 3 store the two chi/2 x
// chi/2 blocks a_0s[q][p] = A[s][2q][2p+s] (s = 0, 1), then the phase
// r = e^{2 i theta_k} that gives the other two, a_1s = r_s a_0s with r_0 = r and
// r_1 = conj(r); reps = 2 stores three unit phases that determine the site.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "../../include/qsvm.h"

namespace qsvm {

constexpr double kPi = 3.14159265358979323846;

// Binary grids of the split-FP32 format.  Tensor and phase hi parts sit on
// 2^-kGridT in every form.  The block-form engine (reps = 1) keeps environment hi
// parts on 2^-kGridE after renormalisation to max |.| < 1, the mixed environment
// G = E_0 + rho E_1 on 2^-kGridG and the intermediate (a^T G) on 2^-grid_x(chi);
// the gauged engines (reps = 2, 3) choose their own grids.  The exactness argument
// (every hi*hi partial sum stays below 2^24 grid units) is spelled out with each
// engine in pair_contract.cuh.
constexpr int kGridT = 11;
constexpr int kGridE = 10;
constexpr int kGridG = 10;
__host__ __device__ constexpr int grid_x(int chi) { return chi >= 8 ? 9 : 10; }

// Site-record geometry, block form (reps = 1; reps = 3 in FP64 and FP32).  A record holds the blocks
// a_00 and a_01 (16 bytes per complex entry) and then the phase entry r.  FP64
// records hold each value once as (re, im).  The FP32 formats hold two forms of
// every record, in two arrays (all row-side "a-form" records of the buffer first,
// then all column-side "b-form" records):
//   a-form entry (A, iA)              = (re, im, -im, re)
//   b-form entry (conj B, i conj B)   = (re, -im, im, re)
// so that a complex multiply-accumulate is two packed FP32x2 FMAs with one
// broadcast operand:  E A = E.re * A + E.im * (iA),  X conj(B) = X.re * conj(B) + X.im * (i conj(B)).
// Split FP32 stores, per block, the hi entries then the lo entries, each in
// form, and the phase as a hi entry then a lo entry.
template <int CHI, int PREC>
struct Record {
  static constexpr int H = CHI / 2;                    // block side
  static constexpr int kEntries = H * H;               // complex entries per block
  static constexpr int kForms = (PREC == QSVM_FP64) ? 1 : 2;
  static constexpr int kEntryBytes = 16;               // (re, im) double, or one form entry of 4 floats
  static constexpr int kParts = (PREC == QSVM_FP32_SPLIT) ? 2 : 1;
  static constexpr int kPartBytes = kEntries * kEntryBytes;
  static constexpr int kBlockBytes = kPartBytes * kParts;
  static constexpr int kBlockStride = kBlockBytes;
  static constexpr int kPhaseOff = 2 * kBlockStride;   // phase r: one entry per part
  static constexpr int kBytes = kPhaseOff + kParts * kEntryBytes;  // one form of one site
};

// Phase form (reps = 2).  With P = e^{-i x_k} and T = e^{-i theta_{k-1}}, the
// site's blocks are a_00 = (1/2) [[P^2 T^2, 1], [P^2, T^2]] and
// a_01 = (1/2) [[1, -conj(P^2 T^2)], [conj(T^2), -conj(P^2)]] (rows q, columns p),
// and r = conj(T^2).  A record holds the three unit phases V_0 = T^2, V_1 = P^2,
// V_2 = P^2 T^2 (the factors 1/2 are carried in the log scale).  Plain FP32 keeps
// them: per value its a-form then its b-form entry (each side of a pair needs both),
// one array.  (FP64 and split FP32 use the gauged form below.)
template <int PREC>
struct Record<4, PREC> {
  static constexpr int H = 2;
  static constexpr int kForms = 1;
  static constexpr int kValBytes = 32;  // one value, both forms
  static constexpr int kBytes = 3 * kValBytes;
  // byte offset of value v (0: T^2, 1: P^2, 2: P^2 T^2), form f (0: a, 1: b)
  __host__ __device__ static constexpr int off(int v, int f) { return v * kValBytes + f * 16; }
};

// Gauged form (split FP32, reps = 2).  A diagonal change of basis on every bond
// leaves the state unchanged; the one that makes the first row (t = 0) of every
// site tensor equal to one turns both blocks of site k into the same matrix
//     a_0s = [[1, 1], [alpha_k, beta_k]],   alpha_k = conj(V_2^{k-1} V_0^k),
//     beta_k = conj(V_2^{k-1}) V_0^k        (V^{k} the phases of site k above),
// with a_1s = r'_s S a_0s, S = diag(1, -1), r'_0 = alpha_k and r'_1 = beta_k
// (and unit-modulus entries: the factors 1/2 stay in the log scale).  The basis
// change left on the last bond is undone by one more, virtual site n with
// alpha_n = beta_n = conj(V_2^{n-1}); the amplitude is then entry (0, 0) of
// block 0 of the environment after site n, up to a phase.  Site 0 (left bond 1)
// stores alpha_0 = beta_0 = 1.  A record holds alpha then beta, each as its hi
// entry then its lo entry; the buffer keeps n + 1 records per point, an a-form
// array (row side) and then a b-form array (column side), so each side of a pair
// reads 64 bytes per site.
// FP64 keeps the same values as (re, im) doubles, alpha then beta (32 bytes), in
// one array of n + 1 records per point: each side conjugates in registers.
template <>
struct Record<4, QSVM_FP64> {
  static constexpr int kForms = 1;
  static constexpr int kBytes = 32;
  __host__ __device__ static constexpr int off(int v) { return v * 16; }
};

template <>
struct Record<4, QSVM_FP32_SPLIT> {
  static constexpr int kForms = 2;
  static constexpr int kBytes = 64;
  // byte offset of value v (0: alpha, 1: beta), part (0: hi, 1: lo) within one form's record
  __host__ __device__ static constexpr int off(int v, int part) { return v * 32 + part * 16; }
};

// Split FP32 and FP64 at reps = 3: the same gauged records as at reps = 2.  The change of
// bond basis that makes row t = 0 of every site one gives, at reps = 3, both blocks
// equal to the signed Kronecker square (-1)^{q1 q2} M[q1][p1] M[q2][p2] of
// M = [[1, 1], [alpha_k, beta_k]] with the alpha_k, beta_k of reps = 2, and the c = 1
// rows r'_s diag(1, 1, -1, -1) times the c = 0 rows (r'_0 = alpha_k, r'_1 = beta_k);
// the virtual site n closes the chain the same way.
template <>
struct Record<8, QSVM_FP32_SPLIT> : Record<4, QSVM_FP32_SPLIT> {};
template <>
struct Record<8, QSVM_FP64> : Record<4, QSVM_FP64> {};

__host__ __device__ constexpr size_t record_bytes(int chi, int prec) {
  return chi == 4 ? (prec == QSVM_FP64 ? 32 : prec == QSVM_FP32 ? 96 : 64)
         : (chi == 8 && prec != QSVM_FP32) ? (prec == QSVM_FP64 ? 32 : 64)
                                                 : (2 * (size_t)(chi / 2) * (chi / 2) + 1) * 16 * (prec == QSVM_FP32_SPLIT ? 2 : 1);
}
static_assert(record_bytes(4, QSVM_FP64) == Record<4, QSVM_FP64>::kBytes, "record geometry");
static_assert(record_bytes(4, QSVM_FP32) == Record<4, QSVM_FP32>::kBytes, "record geometry");
static_assert(record_bytes(4, QSVM_FP32_SPLIT) == Record<4, QSVM_FP32_SPLIT>::kBytes, "record geometry");
static_assert(record_bytes(2, QSVM_FP32) == Record<2, QSVM_FP32>::kBytes, "record geometry");
static_assert(record_bytes(8, QSVM_FP32_SPLIT) == Record<8, QSVM_FP32_SPLIT>::kBytes, "record geometry");
static_assert(record_bytes(8, QSVM_FP64) == Record<8, QSVM_FP64>::kBytes, "record geometry");
static_assert(record_bytes(8, QSVM_FP32) == Record<8, QSVM_FP32>::kBytes, "record geometry");
static_assert(Record<2, QSVM_FP32_SPLIT>::kBytes % 16 == 0 && Record<2, QSVM_FP64>::kBytes % 16 == 0,
              "bulk copies move whole 16-byte units");
// arrays of records a buffer holds (the FP32 block forms and the gauged form keep
// a- and b-form arrays)
__host__ __device__ constexpr int record_forms(int chi, int prec) {
  return (prec == QSVM_FP64 || (chi == 4 && prec == QSVM_FP32)) ? 1 : 2;
}
// records per point and array: one per site, plus the virtual site of the gauged
// form (FP64 and split FP32 at reps = 2 and 3)
__host__ __device__ constexpr int record_sites(int n_qubits, int chi, int prec) {
  return n_qubits + ((chi >= 4 && prec != QSVM_FP32) ? 1 : 0);
}

// ---- tile order --------------------------------------------------------------
// Pair tiles are visited in bands of kBandRows tile rows; within a band column by
// column, within a column row by row.  The CTAs resident at one time then cover a
// few columns of one band, so each column point's site records are fetched from
// DRAM about once per band instead of once per tile row, and a band's row points
// (1024 of them with 16-point tiles: 51 MB of records at n = 784) stay in the L2
// while its columns go by.  At n = 784, N = 8192 this reads 2.9 GB per Gram
// launch against 13.6 GB with bands of 8 tile rows, at the same speed.
constexpr int64_t kBandRows = 64;

// Symmetric Gram (tiles ti <= tj of a T x T grid): tiles before band k (all
// bands before k are full): band m holds G(G+1)/2 + G(T - mG - G) tiles.
__host__ __device__ inline int64_t sym_band_start(int64_t k, int64_t T) {
  const int64_t G = kBandRows;
  return k * (G * (G + 1) / 2 + G * (T - G)) - G * G * k * (k - 1) / 2;
}

__host__ __device__ inline void sym_tile_decode(int64_t b, int64_t T, int64_t& ti, int64_t& tj) {
  const int64_t G = kBandRows;
  int64_t lo = 0, hi = (T + G - 1) / G - 1;  // last band whose start is <= b
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) / 2;
    if (sym_band_start(mid, T) <= b) lo = mid;
    else hi = mid - 1;
  }
  const int64_t r0 = lo * G;
  const int64_t g = (T - r0) < G ? (T - r0) : G;
  int64_t o = b - sym_band_start(lo, T);
  const int64_t tri = g * (g + 1) / 2;
  if (o < tri) {  // the band's triangle: column c holds rows r0 .. r0 + c
    int64_t c = (int64_t)((sqrt(8.0 * (double)o + 1.0) - 1.0) * 0.5);
    while (c > 0 && c * (c + 1) / 2 > o) --c;
    while ((c + 1) * (c + 2) / 2 <= o) ++c;
    tj = r0 + c;
    ti = r0 + (o - c * (c + 1) / 2);
  } else {        // full columns of g tiles each
    o -= tri;
    tj = r0 + g + o / g;
    ti = r0 + o % g;
  }
}

// Cross kernel (Ta x Tb tiles, all of them): bands of G rows, column by column.
__host__ __device__ inline void rect_tile_decode(int64_t b, int64_t Ta, int64_t Tb, int64_t& ti, int64_t& tj) {
  const int64_t G = kBandRows;
  const int64_t k = b / (G * Tb);
  const int64_t r0 = k * G;
  const int64_t g = (Ta - r0) < G ? (Ta - r0) : G;
  const int64_t o = b - k * G * Tb;
  tj = o / g;
  ti = r0 + o % g;
}

// Launch arguments of the per-tile pair kernel.
struct TileArgs {
  const uint8_t* mpsA;   // row points (i): a-form records
  const uint8_t* mpsB;   // column points (j): b-form records
  int64_t nA, nB;
  int n;                 // sites (qubits)
  int symmetric;         // 1: upper-triangle tiles of a Gram (same points on both sides)
  int64_t tile_begin;    // first linear tile index of this launch
  int64_t tiles_i;       // tile rows (cross)
  int64_t tiles_j;       // tile columns (cross) or tiles per side (symmetric)
  double* K;
  int64_t ldk;
  double* logK;          // nullable
  int64_t ldl;
};

// Runtime pipeline configuration of the pair kernels (the autotuner's knobs):
// sites per chunk, number of shared-memory stages in flight, and whether a CTA
// contracts a whole tile or a quarter of one.
struct PipeCfg {
  int S;            // sites per chunk
  int stages;       // 2..4
  int slot_bytes;   // S * record bytes, padded to an odd number of 16-byte units (per point per stage)
  int stage_bytes;  // 2 * tile points * slot_bytes
  int sub;          // 1: a CTA per tile; 2: a CTA per quarter tile
  int tile;         // side of the block of pairs a CTA contracts (tile side / sub)
};

// One Gram job of a batch, as the persistent kernel reads it (64 bytes).
struct DevJob {
  const uint8_t* mps;
  int64_t n_points;
  int64_t tiles;    // tiles per side
  double* K;
  int64_t ldk;
  double* logK;
  int64_t ldl;
  int32_t n_qubits;
  int32_t pad;
};
static_assert(sizeof(DevJob) == 64, "DevJob layout");

struct BatchArgs {
  const DevJob* jobs;
  const int64_t* prefix;            // n_jobs + 1 tile offsets
  unsigned long long* counter;      // work-queue head, zeroed before each launch
  int n_jobs;
  int64_t total_tiles;
};

// ---------------------------------------------------------------- PTX ----
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// One bulk (TMA, untiled) copy global -> shared, completion counted in bytes on
// the mbarrier.  dst, src and bytes must be multiples of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait on an mbarrier phase: true when the phase completed, false after
// `limit_ns` nanoseconds of waiting (the caller then records a timeout).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > limit_ns) return false;
  }
}

constexpr uint64_t kWaitLimitNs = 4000000000ull;    // 4 s: a chunk copy takes microseconds
constexpr uint64_t kDrainLimitNs = 1000000000ull;   // after a timeout, wait at most 1 s more

// ----------------------------------------------------------- scalars -----
// Exact scaling by 2^-e for |e| <= 126 (single power-of-two multiply).
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((127 + e) << 23); }
__device__ __forceinline__ double pow2d(int e) { return __longlong_as_double((long long)(1023 + e) << 52); }

// Round to the nearest multiple of 2^-g (ties to even) without leaving FP32:
// (v + 1.5*2^(23-g)) - 1.5*2^(23-g), valid for |v| < 2^(22-g).
template <int G>
__device__ __forceinline__ float grid_round(float v) {
  constexpr float C = 1.5f * (float)(1 << (23 - G));
  return __fsub_rn(__fadd_rn(v, C), C);
}

}  // namespace qsvm
