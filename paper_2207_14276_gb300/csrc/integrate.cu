// Velocity-Verlet kick and drift for the multiple-time-step driver that calls
// the potential on the ML region every outer step (paper Eq. 7 and the RESPA
// scheme of the hybrid simulations): v += dt_kick a, then x += dt_drift v, over
// the atoms of the mask, with the kinetic energy of those atoms reduced in FP64.
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/nnp.h"

namespace {

// 1 kcal/mol/A per g/mol, in A/fs^2
constexpr double kAccel = 4.184e-4;

__global__ void k_integrate(int n, float* __restrict__ x, float* __restrict__ v,
                            const float* __restrict__ f, const float* __restrict__ inv_m,
                            const uint8_t* __restrict__ mask, float ck, float dd,
                            double* __restrict__ ke) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double e = 0.0;
  if (i < n && (!mask || mask[i])) {
    const float im = inv_m[i];
    float v2 = 0.f;
    for (int c = 0; c < 3; ++c) {
      const float vc = fmaf(ck * im, f ? f[3 * i + c] : 0.f, v[3 * i + c]);
      v[3 * i + c] = vc;
      x[3 * i + c] = fmaf(dd, vc, x[3 * i + c]);
      v2 = fmaf(vc, vc, v2);
    }
    e = im > 0.f ? 0.5 * (double)v2 / ((double)im * kAccel) : 0.0;
  }
  if (!ke) return;
  for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
  if ((threadIdx.x & 31) == 0 && e != 0.0) atomicAdd(ke, e);
}

}  // namespace

extern "C" int nnp_integrate(int64_t n_atoms, float* coords, float* velocities,
                             const float* forces, const float* inv_masses, const uint8_t* mask,
                             float dt_kick_fs, float dt_drift_fs, double* kinetic, void* stream) {
  if (n_atoms < 0 || n_atoms > (1LL << 30)) return NNP_ERR_ARG;
  if (n_atoms > 0 && (!coords || !velocities || !inv_masses)) return NNP_ERR_ARG;
  if (!(dt_kick_fs == dt_kick_fs) || !(dt_drift_fs == dt_drift_fs)) return NNP_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (kinetic && cudaMemsetAsync(kinetic, 0, sizeof(double), st) != cudaSuccess) return NNP_ERR_CUDA;
  if (n_atoms == 0) return NNP_OK;
  const int n = (int)n_atoms;
  k_integrate<<<(n + 255) / 256, 256, 0, st>>>(n, coords, velocities, forces, inv_masses, mask,
                                               (float)(dt_kick_fs * kAccel), dt_drift_fs, kinetic);
  return cudaGetLastError() == cudaSuccess ? NNP_OK : NNP_ERR_CUDA;
}
