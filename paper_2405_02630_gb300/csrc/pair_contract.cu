// pair_contract.cu -- launchers of the pair-contraction kernels (see pair_contract.cuh).
#include <climits>

#include "pair_contract.cuh"

namespace qsvm {

template <int CHI, int PREC>
static cudaError_t launch_pair_t(const TileArgs& a, int64_t ntiles, cudaStream_t st) {
  using Cfg = TileCfg<CHI, PREC>;
  auto kern = pair_tile_kernel<CHI, PREC>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::kSmem);
  if (e != cudaSuccess) return e;
  int64_t done = 0;
  while (done < ntiles) {
    const int64_t cnt = (ntiles - done) < (int64_t)INT_MAX ? (ntiles - done) : (int64_t)INT_MAX;
    TileArgs b = a;
    b.tile_begin = a.tile_begin + done;
    kern<<<(unsigned)cnt, Cfg::TI * Cfg::TI, Cfg::kSmem, st>>>(b);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    done += cnt;
  }
  return cudaSuccess;
}

template <int CHI>
static cudaError_t launch_pair_c(int prec, const TileArgs& a, int64_t ntiles, cudaStream_t st) {
  switch (prec) {
    case QSVM_FP64: return launch_pair_t<CHI, QSVM_FP64>(a, ntiles, st);
    case QSVM_FP32: return launch_pair_t<CHI, QSVM_FP32>(a, ntiles, st);
    default: return launch_pair_t<CHI, QSVM_FP32_SPLIT>(a, ntiles, st);
  }
}

cudaError_t launch_pair(int chi, int prec, const TileArgs& a, int64_t ntiles, cudaStream_t st) {
  switch (chi) {
    case 2: return launch_pair_c<2>(prec, a, ntiles, st);
    case 4: return launch_pair_c<4>(prec, a, ntiles, st);
    default: return launch_pair_c<8>(prec, a, ntiles, st);
  }
}

int pair_tile_dim(int chi, int prec) {
  (void)chi;
  (void)prec;
  return TileCfg<4, QSVM_FP64>::TI;
}

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
