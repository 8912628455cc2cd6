// Device build of the CUDA path's per-particle arithmetic (csrc/collapse.cuh)
// behind a host function, so that GPU tests can compare it with the oracle
// one particle at a time.
#include <cuda_runtime.h>

#include "collapse.cuh"

__global__ void k_eval(const double* lam, const double* h, int n, int corr, double dcorr, int use_float,
                       double* F, double* kap, double* eig) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
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
