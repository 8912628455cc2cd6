// Host build of the CUDA path's per-particle eigenvalue and collapse arithmetic
// (csrc/collapse.cuh), so that tests can compare it with the oracle on the CPU.
#include <cstdio>
#include <cstdlib>
#include "collapse.cuh"
extern "C" double host_collapse(const double* lam, int corr, int use_float, double dcorr, double* kap) {
  if (use_float) {
    float l[3] = {(float)lam[0], (float)lam[1], (float)lam[2]};
    pin::CollapseConsts<float> cc{(float)dcorr, corr};
    float k; float F = pin::collapse_from_eigs<float>(l, cc, k); *kap = k; return F;
  }
  pin::CollapseConsts<double> cc{dcorr, corr};
  double k; double F = pin::collapse_from_eigs<double>(lam, cc, k); *kap = k; return F;
}
extern "C" double host_eig(const double* h, double* lam, int use_float) {
  if (use_float) { float hf[6], lf[3]; for (int i=0;i<6;++i) hf[i]=(float)h[i]; float r = pin::eig3<float>(hf, lf); for(int i=0;i<3;++i) lam[i]=lf[i]; return r; }
  return pin::eig3<double>(h, lam);
}
extern "C" double host_bound(const double* h, int corr, int use_float, double dcorr) {
  if (use_float) {
    float hf[6];
    for (int i = 0; i < 6; ++i) hf[i] = (float)h[i];
    pin::CollapseConsts<float> cc{(float)dcorr, corr};
    return pin::collapse_bound<float>(hf, cc);
  }
  pin::CollapseConsts<double> cc{dcorr, corr};
  return pin::collapse_bound<double>(h, cc);
}
