// Seeded initial conditions generated on the device (pin_set_ic_seed): the
// same counter-based generator as the host module (include/pin_ic.h: P(k) =
// A k^ns T_BBKS(k/Gamma)^2, splitmix64 keyed on (seed, linear mode index),
// Box-Muller, Hermitian symmetry on the kz = 0 and kz = N/2 planes), each mode
// computed independently in FP64 with the device's own math functions and
// cast to FP32.  It produces inputs only, none of the collapse arithmetic.
#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.cuh"

namespace pin {
namespace {

constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ULL;

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + kGolden;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

__device__ __forceinline__ double bbks(double q) {
  if (q <= 0.0) return 1.0;
  const double a = 2.34 * q;
  const double lead = log(1.0 + a) / a;
  // explicit rounded product: no fused multiply-add, as in the host build
  const double p = 1.0 + __dmul_rn(3.89, q) + pow(16.1 * q, 2.0) + pow(5.46 * q, 3.0) + pow(6.71 * q, 4.0);
  return lead * pow(p, -0.25);
}

__device__ __forceinline__ void mode_value(int n, double box, uint64_t key, double amp, double ns, double gamma,
                                           int ix, int iy, int iz, double* re, double* im) {
  const int nh = n / 2 + 1;
  const double sx = ix < n / 2 ? ix : ix - n, sy = iy < n / 2 ? iy : iy - n;
  const double sz = iz < n / 2 ? iz : -(n / 2);
  const double kk = 2.0 * M_PI / box * sqrt(sx * sx + sy * sy + sz * sz);
  double P = 0.0;
  if (kk > 0.0) {
    const double t = bbks(kk / gamma);
    P = amp * pow(kk, ns) * t * t;
  }
  const double scale = sqrt((double)n * n * n * (double)n * n * n * P / (box * box * box));
  const uint64_t m = ((uint64_t)ix * n + iy) * nh + iz;
  const uint64_t r1 = splitmix64(key + (2 * m + 1) * kGolden);
  const uint64_t r2 = splitmix64(key + (2 * m + 2) * kGolden);
  const double u1 = ((double)((r1 >> 11) + 1)) * 0x1.0p-53;  // (0, 1]
  const double u2 = ((double)(r2 >> 11)) * 0x1.0p-53;        // [0, 1)
  const double rad = sqrt(-2.0 * log(u1));
  *re = scale * (rad * cos(2.0 * M_PI * u2)) / sqrt(2.0);
  *im = scale * (rad * sin(2.0 * M_PI * u2)) / sqrt(2.0);
}

// One realisation per blockIdx.y; out holds batch half-spectra [n][n][n/2+1].
__global__ void k_ic_seed(int n, double box, const uint64_t* keys, double amp, double ns, double gamma,
                          float2* out) {
  const int nh = n / 2 + 1;
  const size_t total = (size_t)n * n * nh;
  const uint64_t key = keys[blockIdx.y];
  float2* o = out + (size_t)blockIdx.y * total;
  for (size_t m = blockIdx.x * (size_t)blockDim.x + threadIdx.x; m < total; m += (size_t)gridDim.x * blockDim.x) {
    const int iz = (int)(m % nh);
    const size_t r = m / nh;
    const int iy = (int)(r % n), ix = (int)(r / n);
    double re = 0.0, im = 0.0;
    if (!(ix == 0 && iy == 0 && iz == 0)) {
      if (iz == 0 || iz == n / 2) {
        const int jx = (n - ix) % n, jy = (n - iy) % n;
        const size_t mm = ((size_t)jx * n + jy) * nh + iz;
        if (mm == m) {
          mode_value(n, box, key, amp, ns, gamma, ix, iy, iz, &re, &im);
          re *= sqrt(2.0);
          im = 0.0;
        } else if (mm < m) {
          mode_value(n, box, key, amp, ns, gamma, jx, jy, iz, &re, &im);
          im = -im;
        } else {
          mode_value(n, box, key, amp, ns, gamma, ix, iy, iz, &re, &im);
        }
      } else {
        mode_value(n, box, key, amp, ns, gamma, ix, iy, iz, &re, &im);
      }
    }
    o[m] = make_float2((float)re, (float)im);
  }
}

}  // namespace

cudaError_t generate_ic(int n, double box, const uint64_t* keys_dev, int batch, double amp, double ns,
                        double gamma, float2* out, cudaStream_t st) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t total = (size_t)n * n * (n / 2 + 1);
  const size_t want = (total + 255) / 256;
  const unsigned gx = (unsigned)(want < (size_t)sms * 16 ? want : (size_t)sms * 16);
  k_ic_seed<<<dim3(gx, (unsigned)batch), 256, 0, st>>>(n, box, keys_dev, amp, ns, gamma, out);
  return cudaGetLastError();
}

}  // namespace pin
