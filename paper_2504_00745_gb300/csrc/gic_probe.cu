// gic_probe.cu -- measurement aids: the FMA rate of this GPU in FP32 and
// FP64 (the ceiling of arithmetic-bound kernels, against which the FP64
// path's throughput is read).  No counterpart in the paper.
#include "gic_internal.cuh"

namespace gic {

constexpr int kProbeThreads = 256;
constexpr int kProbeChains = 8;

// kProbeChains independent FMA chains per thread, iters steps each; the sum
// is stored so that nothing is optimised away.
template <typename T>
__global__ void __launch_bounds__(kProbeThreads) k_probe_fma(int iters, T* __restrict__ sink) {
  T a[kProbeChains];
  const T b = T(0.9999999), c = T(1e-7);
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) a[k] = T(threadIdx.x + k) * T(1e-3);
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) a[k] = fma(a[k], b, c);
  T s = T(0);
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) s += a[k];
  sink[blockIdx.x * (int64_t)kProbeThreads + threadIdx.x] = s;
}

}  // namespace gic

using namespace gic;

extern "C" int gic_probe_fma(int32_t precision, int32_t blocks, int32_t iters, void* sink, int64_t* fmas,
                             gic_stream_t stream) {
  GIC_RANGE("gic_probe_fma");
  if (precision != GIC_FP32 && precision != GIC_FP64)
    return set_error(GIC_ERR_INVALID, "gic_probe_fma: unknown precision %d", (int)precision);
  if (blocks < 1 || iters < 1) return set_error(GIC_ERR_INVALID, "gic_probe_fma: blocks and iters must be >= 1");
  if (!sink) return set_error(GIC_ERR_INVALID, "gic_probe_fma: sink is NULL");
  if ((uintptr_t)sink % 8) return set_error(GIC_ERR_ALIGN, "gic_probe_fma: sink must be 8-byte aligned");
  if (precision == GIC_FP32)
    k_probe_fma<float><<<blocks, kProbeThreads, 0, (cudaStream_t)stream>>>(iters, (float*)sink);
  else
    k_probe_fma<double><<<blocks, kProbeThreads, 0, (cudaStream_t)stream>>>(iters, (double*)sink);
  count_launches(1);
  if (fmas) *fmas = (int64_t)blocks * kProbeThreads * kProbeChains * (int64_t)iters;
  GIC_CHECK_LAUNCH("gic_probe_fma");
  return GIC_OK;
}
