// pair_contract.cu -- launchers of the pair-contraction kernels (see pair_contract.cuh).
#include <climits>

#include "pair_contract.cuh"

namespace qsvm {

// Candidate pipeline shapes the autotuner chooses from: bytes of site records per
// point and chunk, and stages in flight (default_shape() picks per chi and precision).
struct PipeShape {
  int chunk_bytes;
  int stages;
};
static const PipeShape kShapes[] = {{512, 4},  {1024, 3}, {512, 3},  {1024, 2}, {1024, 4},  {2048, 2},
                                    {2048, 3}, {512, 2},  {1152, 2}, {1440, 2}, {2304, 2}, {3456, 2}};
constexpr int kNumShapes = (int)(sizeof(kShapes) / sizeof(kShapes[0]));
// Configurations: shape c % kNumShapes with whole tiles per CTA (c < kNumShapes)
// or a quarter tile per CTA (c >= kNumShapes).
constexpr int kNumSubs = 2;

// Defaults from shape sweeps on one GB300 (n = 784 Grams): split FP32 with 64-byte
// gauged records, two stages of 22 sites at reps = 2 and of 32 sites at reps = 3
// (each within 0.5 % of the best of the twelve shapes); plain FP32 two stages of
// fifteen phase-form sites.  FP64 is insensitive (within 0.3 %).  Two stages keep
// two CTAs per SM and the longer chunks pay the per-chunk wait and hand-off less
// often.
int default_shape(int chi, int prec) {
  if (chi == 4 && prec == QSVM_FP32_SPLIT) return 9;
  if (chi == 4 && prec == QSVM_FP32) return 9;
  if (chi >= 8 && prec == QSVM_FP32_SPLIT) return 5;
  return (prec == QSVM_FP32 || chi >= 8) ? 3 : 1;
}

int num_pipe_shapes() { return kNumShapes * kNumSubs; }

PipeCfg make_pipe(int chi, int prec, int config) {
  int shape = config, sub = 1;
  if (config < 0 || config >= kNumShapes * kNumSubs) {
    shape = default_shape(chi, prec);
  } else {
    shape = config % kNumShapes;
    sub = 1 + config / kNumShapes;
  }
  const int rec = (int)record_bytes(chi, prec);
  PipeCfg pc;
  pc.S = kShapes[shape].chunk_bytes >= rec ? kShapes[shape].chunk_bytes / rec : 1;
  pc.stages = kShapes[shape].stages;
  // A warp's lanes read 16-byte entries of up to 16 points' slots at once.  A slot
  // stride that is an odd number of 16-byte units puts 8 consecutive slots in the
  // 8 different 16-byte bank groups of a 128-byte row, so those reads take the
  // minimum number of wavefronts (an even stride, e.g. 7 FP32 sites = 1008 + 16
  // bytes, sends all 16 lanes to one group).
  pc.slot_bytes = pc.S * rec;
  if ((pc.slot_bytes / 16) % 2 == 0) pc.slot_bytes += 16;
  pc.sub = sub;
  pc.tile = tile_side(chi, prec) / sub;
  pc.stage_bytes = 2 * pc.tile * pc.slot_bytes;
  return pc;
}

// The persistent batch kernel always contracts whole tiles: the same shape with sub = 1.
PipeCfg whole_tile_pipe(int chi, int prec, int config) {
  return make_pipe(chi, prec, (config < 0 || config >= kNumShapes * kNumSubs) ? -1 : config % kNumShapes);
}

int pipe_smem(const PipeCfg& pc, int chi, int prec) { return pipe_smem_bytes(pc, chi, prec); }

template <int CHI, int PREC, int SUB>
static cudaError_t launch_pair_sub(const TileArgs& a, int64_t ntiles, const PipeCfg& pc, cudaStream_t st) {
  auto kern = pair_tile_kernel<CHI, PREC, SUB>;
  const int smem = pipe_smem_bytes(pc, CHI, PREC);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const int64_t per_launch = (int64_t)INT_MAX / (SUB * SUB);  // tiles per launch: grid = SUB^2 x tiles
  int64_t done = 0;
  while (done < ntiles) {
    const int64_t cnt = (ntiles - done) < per_launch ? (ntiles - done) : per_launch;
    TileArgs b = a;
    b.tile_begin = a.tile_begin + done;
    kern<<<(unsigned)(cnt * SUB * SUB), kernel_threads<CHI, PREC, SUB>(), smem, st>>>(b, pc);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    done += cnt;
  }
  return cudaSuccess;
}

template <int CHI, int PREC>
static cudaError_t launch_pair_t(const TileArgs& a, int64_t ntiles, const PipeCfg& pc, cudaStream_t st) {
  return pc.sub == 2 ? launch_pair_sub<CHI, PREC, 2>(a, ntiles, pc, st) : launch_pair_sub<CHI, PREC, 1>(a, ntiles, pc, st);
}

// Sets the kernel's shared-memory attribute and sizes its grid (SMs x resident
// CTAs per SM, at most one CTA per tile).  Kept out of the launch so a launch can
// be recorded in a CUDA graph without attribute or occupancy calls inside it.
template <int CHI, int PREC>
static cudaError_t prepare_persistent_t(const PipeCfg& pc, int64_t total_tiles, int* grid_out) {
  auto kern = pair_persistent_kernel<CHI, PREC>;
  const int smem = pipe_smem_bytes(pc, CHI, PREC);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kernel_threads<CHI, PREC, 1>(), smem)) !=
      cudaSuccess)
    return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  int64_t grid = (int64_t)sms * per_sm;
  if (grid > total_tiles) grid = total_tiles;
  *grid_out = (int)(grid < 1 ? 1 : grid);
  return cudaSuccess;
}

template <int CHI, int PREC>
static cudaError_t launch_persistent_t(const BatchArgs& a, const PipeCfg& pc, int grid, cudaStream_t st) {
  pair_persistent_kernel<CHI, PREC><<<(unsigned)grid, kernel_threads<CHI, PREC, 1>(), pipe_smem_bytes(pc, CHI, PREC),
                                      st>>>(a, pc);
  return cudaGetLastError();
}

template <int CHI>
static cudaError_t launch_pair_c(int prec, const TileArgs& a, int64_t ntiles, const PipeCfg& pc, cudaStream_t st) {
  switch (prec) {
    case QSVM_FP64: return launch_pair_t<CHI, QSVM_FP64>(a, ntiles, pc, st);
    case QSVM_FP32: return launch_pair_t<CHI, QSVM_FP32>(a, ntiles, pc, st);
    default: return launch_pair_t<CHI, QSVM_FP32_SPLIT>(a, ntiles, pc, st);
  }
}

template <int CHI>
static cudaError_t prepare_persistent_c(int prec, const PipeCfg& pc, int64_t total, int* g) {
  switch (prec) {
    case QSVM_FP64: return prepare_persistent_t<CHI, QSVM_FP64>(pc, total, g);
    case QSVM_FP32: return prepare_persistent_t<CHI, QSVM_FP32>(pc, total, g);
    default: return prepare_persistent_t<CHI, QSVM_FP32_SPLIT>(pc, total, g);
  }
}

template <int CHI>
static cudaError_t launch_persistent_c(int prec, const BatchArgs& a, const PipeCfg& pc, int grid, cudaStream_t st) {
  switch (prec) {
    case QSVM_FP64: return launch_persistent_t<CHI, QSVM_FP64>(a, pc, grid, st);
    case QSVM_FP32: return launch_persistent_t<CHI, QSVM_FP32>(a, pc, grid, st);
    default: return launch_persistent_t<CHI, QSVM_FP32_SPLIT>(a, pc, grid, st);
  }
}

cudaError_t launch_pair(int chi, int prec, const TileArgs& a, int64_t ntiles, const PipeCfg& pc, cudaStream_t st) {
  switch (chi) {
    case 2: return launch_pair_c<2>(prec, a, ntiles, pc, st);
    case 4: return launch_pair_c<4>(prec, a, ntiles, pc, st);
    default: return launch_pair_c<8>(prec, a, ntiles, pc, st);
  }
}

cudaError_t prepare_persistent(int chi, int prec, const PipeCfg& pc, int64_t total_tiles, int* grid_out) {
  switch (chi) {
    case 2: return prepare_persistent_c<2>(prec, pc, total_tiles, grid_out);
    case 4: return prepare_persistent_c<4>(prec, pc, total_tiles, grid_out);
    default: return prepare_persistent_c<8>(prec, pc, total_tiles, grid_out);
  }
}

cudaError_t launch_persistent(int chi, int prec, const BatchArgs& a, const PipeCfg& pc, int grid, cudaStream_t st) {
  switch (chi) {
    case 2: return launch_persistent_c<2>(prec, a, pc, grid, st);
    case 4: return launch_persistent_c<4>(prec, a, pc, grid, st);
    default: return launch_persistent_c<8>(prec, a, pc, grid, st);
  }
}

int pair_tile_dim(int chi, int prec) { return tile_side(chi, prec); }
int pair_threads(int chi, int prec) { return threads_per_pair(chi, prec); }

cudaError_t pair_status(cudaStream_t st, int clear, int32_t* out) {
  int32_t v = 0;
  cudaError_t e = cudaMemcpyFromSymbolAsync(&v, g_pair_status, sizeof(int32_t), 0, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess && clear) {
    const int32_t z = 0;
    e = cudaMemcpyToSymbolAsync(g_pair_status, &z, sizeof(int32_t), 0, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  *out = v;
  return e;
}

}  // namespace qsvm

namespace qsvm {

// Failure-path self test: one CTA waits on an mbarrier phase that nothing will
// complete (no thread arrives, no copy is issued), with a caller-given bound.
// The bounded wait gives up, the kernel records QSVM_ERR_TIMEOUT in the status
// word exactly as a pair kernel does, and returns; the context stays usable.
__global__ void wait_timeout_selftest_kernel(uint64_t limit_ns) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  const bool ok = mbar_wait_bounded(&bar, 0u, limit_ns);
  if (!ok && threadIdx.x == 0) atomicCAS(&g_pair_status, 0, (int32_t)QSVM_ERR_TIMEOUT);
}

cudaError_t launch_wait_timeout_selftest(uint64_t limit_ns, cudaStream_t st) {
  wait_timeout_selftest_kernel<<<1, 32, 0, st>>>(limit_ns);
  return cudaGetLastError();
}

}  // namespace qsvm
