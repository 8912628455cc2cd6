// Device build of the CUDA path's per-particle arithmetic (csrc/collapse.cuh,
// and the two-particle packed form of csrc/collapse_x2.cuh) behind a host
// function, so that GPU tests can compare it with the oracle particle by
// particle.  use_float: 0 FP64, 1 FP32 one particle per thread, 2 FP32 packed
// pairs (thread i evaluates particles i and i + n/2, n even).
#include <cuda_runtime.h>

#include "collapse.cuh"
#include "collapse_x2.cuh"

__global__ void k_eval(const double* lam, const double* h, int n, int corr, double dcorr, int use_float,
                       double* F, double* kap, double* eig) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (use_float == 2) {
    const int m = n / 2;
    if (i >= m) return;
    const int j[2] = {i, i + m};
    float2 l[3], hf[6], le[3];
    for (int k = 0; k < 3; ++k) l[k] = make_float2((float)lam[3 * j[0] + k], (float)lam[3 * j[1] + k]);
    for (int k = 0; k < 6; ++k) hf[k] = make_float2((float)h[6 * j[0] + k], (float)h[6 * j[1] + k]);
    pin::CollapseConsts<float> cc{(float)dcorr, corr};
    float2 k2;
    const float2 f = pin::collapse_from_eigs_x2(l, cc, k2);
    F[j[0]] = f.x;
    F[j[1]] = f.y;
    kap[j[0]] = k2.x;
    kap[j[1]] = k2.y;
    pin::eig3_x2(hf, le);
    for (int k = 0; k < 3; ++k) {
      eig[3 * j[0] + k] = le[k].x;
      eig[3 * j[1] + k] = le[k].y;
    }
    return;
  }
  if (i >= n) return;
  if (use_float) {
    float l[3] = {(float)lam[3 * i], (float)lam[3 * i + 1], (float)lam[3 * i + 2]};
    pin::CollapseConsts<float> cc{(float)dcorr, corr};
    float k;
    F[i] = pin::collapse_from_eigs<float>(l, cc, k);
    kap[i] = k;
    float hf[6], le[3];
    for (int j = 0; j < 6; ++j) hf[j] = (float)h[6 * i + j];
    pin::eig3<float>(hf, le);
    for (int j = 0; j < 3; ++j) eig[3 * i + j] = le[j];
  } else {
    pin::CollapseConsts<double> cc{dcorr, corr};
    double k;
    F[i] = pin::collapse_from_eigs<double>(lam + 3 * i, cc, k);
    kap[i] = k;
    pin::eig3<double>(h + 6 * i, eig + 3 * i);
  }
}

extern "C" int dev_eval(const double* lam, const double* h, int n, int corr, double dcorr, int use_float,
                        double* F, double* kap, double* eig) {
  double *dl, *dh, *dF, *dk, *de;
  if (cudaMalloc(&dl, 24 * n) || cudaMalloc(&dh, 48 * n) || cudaMalloc(&dF, 8 * n) ||
      cudaMalloc(&dk, 8 * n) || cudaMalloc(&de, 24 * n))
    return 1;
  cudaMemcpy(dl, lam, 24 * n, cudaMemcpyHostToDevice);
  cudaMemcpy(dh, h, 48 * n, cudaMemcpyHostToDevice);
  k_eval<<<(n + 127) / 128, 128>>>(dl, dh, n, corr, dcorr, use_float, dF, dk, de);
  int rc = cudaDeviceSynchronize() != cudaSuccess;
  cudaMemcpy(F, dF, 8 * n, cudaMemcpyDeviceToHost);
  cudaMemcpy(kap, dk, 8 * n, cudaMemcpyDeviceToHost);
  cudaMemcpy(eig, de, 24 * n, cudaMemcpyDeviceToHost);
  cudaFree(dl); cudaFree(dh); cudaFree(dF); cudaFree(dk); cudaFree(de);
  return rc;
}
