// qds_inputs.cu -- per-step currents of the driven benchmark workloads, made
// on the device: uniform noise on every component, mode and cell plus the
// stationary m = 0 bunch current j_x.  This is synthetic input, not part of
// the scheme; it lives here so that a step's currents cost one kernel.
//
// Random numbers: SplitMix64 (Steele, Lea and Flood, "Fast splittable
// pseudorandom number generators", OOPSLA 2014), counter-based: the value of
// element e of step n is mix(key(seed, n) + e), so any step can be redrawn
// alone and the draw does not depend on the launch shape.  The noise values
// are FP32 numbers (the same in FP32 and FP64 runs); the bunch is added in
// FP64 and the sum rounded once to the working precision.
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "../../include/qds.h"

void qds_internal_set_error(const std::string &m);  // defined in qds_api.cu

namespace {

__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// uniform in [-amp, amp): u, the top 24 bits of z, gives u 2^-23 - 1 in
// [-1, 1) exactly in FP32, scaled by amp (FP32, one rounding).  The value is
// the same whatever the working precision (FP64 runs see it widened).
__device__ __forceinline__ float sym_noise(uint64_t z, float amp) {
  return amp * ((float)(unsigned)(z >> 40) * 0x1.0p-23f - 1.0f);
}

// grid: x over the elements of one step (32-bit indices: a step's three
// components hold fewer than 2^31 elements), y over the steps
template <class T2>
__global__ void bunch_currents_kernel(T2 *jx, T2 *jr, T2 *jth, int M, int nx, int nr, uint64_t seed_key,
                                      unsigned long long step0, int count, float amp, const double *bunch) {
  const unsigned xr = (unsigned)nx * (unsigned)nr, plane = (unsigned)M * xr, per_step = 3u * plane;
  for (int k = blockIdx.y; k < count; k += gridDim.y) {
    const uint64_t key = splitmix64(seed_key ^ (step0 + (unsigned long long)k));
    const size_t base = (size_t)k * plane;
    for (unsigned e = blockIdx.x * blockDim.x + threadIdx.x; e < per_step; e += gridDim.x * blockDim.x) {
      const unsigned c = e / plane;        // component j_x, j_r, j_theta
      const unsigned q = e - c * plane;    // [m][x][r]
      const unsigned m = q / xr;
      const float re = sym_noise(splitmix64(key + 2 * (uint64_t)e), amp);
      const float im = m == 0 ? 0.0f : sym_noise(splitmix64(key + 2 * (uint64_t)e + 1), amp);
      T2 v;
      if (c == 0 && m == 0 && bunch) v.x = (double)re + bunch[q];  // FP64 sum, rounded once to the output
      else v.x = re;
      v.y = im;
      (c == 0 ? jx : c == 1 ? jr : jth)[base + q] = v;
    }
  }
}

}  // namespace

extern "C" int qds_bunch_currents(int n_modes, int nx, int nr, unsigned long long seed, unsigned long long step,
                                  int count, double amp, const double *bunch_dev, void *jx_dev, void *jr_dev,
                                  void *jth_dev, int fp32, void *stream) {
  if (n_modes < 1 || nx < 1 || nr < 1 || count < 0 || (count > 0 && (!jx_dev || !jr_dev || !jth_dev))) {
    qds_internal_set_error("bunch currents: bad sizes or NULL output");
    return QDS_ERR_INVALID_ARG;
  }
  if (count == 0) return QDS_OK;
  const long long per_step = 3LL * n_modes * nx * nr;
  if (per_step >= (1LL << 31)) {
    qds_internal_set_error("bunch currents: more than 2^31 elements per step");
    return QDS_ERR_INVALID_ARG;
  }
  const uint64_t seed_key = splitmix64(seed);
  const int threads = 256;
  const long long want = (per_step + threads - 1) / threads;
  const dim3 blocks((unsigned)(want < 1184 ? want : 1184), (unsigned)(count < 65535 ? count : 65535));
  cudaStream_t st = (cudaStream_t)stream;
  if (fp32)
    bunch_currents_kernel<float2><<<blocks, threads, 0, st>>>((float2 *)jx_dev, (float2 *)jr_dev, (float2 *)jth_dev,
                                                              n_modes, nx, nr, seed_key, step, count, amp, bunch_dev);
  else
    bunch_currents_kernel<double2><<<blocks, threads, 0, st>>>((double2 *)jx_dev, (double2 *)jr_dev,
                                                               (double2 *)jth_dev, n_modes, nx, nr, seed_key, step,
                                                               count, amp, bunch_dev);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    qds_internal_set_error(std::string("bunch currents launch: ") + cudaGetErrorString(e));
    return QDS_ERR_CUDA;
  }
  return QDS_OK;
}
