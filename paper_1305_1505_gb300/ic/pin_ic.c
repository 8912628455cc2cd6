/*
 * Seeded synthetic Gaussian initial conditions (declared in include/pin_ic.h).
 *
 * The paper draws its linear field with N-GenIC (Sec. 2.2) for a cosmology
 * normalised to sigma8 under top-hat smoothing at 8 Mpc/h (Sec. 2.1.1).  This
 * file is an input generator only: it is consumed identically by the CUDA path,
 * by the CPU oracle and by the benchmark, and holds none of the collapse-time
 * arithmetic.
 */
#include "pin_ic.h"

#include <math.h>
#include <stddef.h>

#define GOLDEN_GAMMA 0x9E3779B97F4A7C15ULL

uint64_t pin_ic_splitmix64(uint64_t x) {
  /* splitmix64 (Steele, Lea & Flood 2014): advance by the golden gamma, then
   * the variant-13 finaliser. */
  uint64_t z = x + GOLDEN_GAMMA;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

double pin_ic_bbks(double q) {
  /* Bardeen, Bond, Kaiser & Szalay 1986, Eq. (G3), adiabatic CDM. */
  if (q <= 0.0) return 1.0;
  double a = 2.34 * q;
  double lead = log(1.0 + a) / a;
  double p = 1.0 + 3.89 * q + pow(16.1 * q, 2) + pow(5.46 * q, 3) + pow(6.71 * q, 4);
  return lead * pow(p, -0.25);
}

double pin_ic_power(double k, const pin_spectrum* ps, double amplitude) {
  if (k <= 0.0) return 0.0;
  double t = pin_ic_bbks(k / ps->gamma);
  return amplitude * pow(k, ps->ns) * t * t;
}

static double tophat_window(double x) {
  /* Fourier transform of a unit top-hat sphere, 3 (sin x - x cos x) / x^3. */
  if (x < 1e-3) return 1.0 - x * x / 10.0;
  return 3.0 * (sin(x) - x * cos(x)) / (x * x * x);
}

double pin_ic_amplitude(const pin_spectrum* ps) {
  /* sigma^2(R) = 1/(2 pi^2) int P(k) W(kR)^2 k^3 dln k, Simpson with 2^16
   * intervals over ln k in [ln 1e-5, ln 1e3], for A = 1, R = 8 Mpc/h. */
  const int nint = 1 << 16;
  const double lo = log(1e-5), hi = log(1e3);
  const double h = (hi - lo) / nint;
  double sum = 0.0;
  for (int i = 0; i <= nint; ++i) {
    double lk = lo + h * i;
    double k = exp(lk);
    double w = tophat_window(k * 8.0);
    double f = pin_ic_power(k, ps, 1.0) * w * w * k * k * k;
    double c = (i == 0 || i == nint) ? 1.0 : ((i & 1) ? 4.0 : 2.0);
    sum += c * f;
  }
  double sigma2 = sum * h / 3.0 / (2.0 * M_PI * M_PI);
  return ps->sigma8 * ps->sigma8 / sigma2;
}

static int signed_index(int i, int n) { return i < n / 2 ? i : i - n; }

/* Unconstrained complex Gaussian draw for linear mode index m (unit variance
 * of |g|^2 / 2 per component pair, i.e. <|g1 + i g2|^2> = 2). */
static void draw_pair(uint64_t key, uint64_t m, double* g1, double* g2) {
  uint64_t r1 = pin_ic_splitmix64(key + (2 * m + 1) * GOLDEN_GAMMA);
  uint64_t r2 = pin_ic_splitmix64(key + (2 * m + 2) * GOLDEN_GAMMA);
  double u1 = ((double)((r1 >> 11) + 1)) * 0x1.0p-53; /* (0, 1] */
  double u2 = ((double)(r2 >> 11)) * 0x1.0p-53;       /* [0, 1) */
  double rad = sqrt(-2.0 * log(u1));
  *g1 = rad * cos(2.0 * M_PI * u2);
  *g2 = rad * sin(2.0 * M_PI * u2);
}

static void mode_value(int n, double box, uint64_t key, const pin_spectrum* ps,
                       double amp, int ix, int iy, int iz, double* re, double* im) {
  const int nh = n / 2 + 1;
  double sx = signed_index(ix, n), sy = signed_index(iy, n);
  double sz = (iz < n / 2) ? iz : -(n / 2);
  double kk = 2.0 * M_PI / box * sqrt(sx * sx + sy * sy + sz * sz);
  double scale = sqrt((double)n * n * n * (double)n * n * n * pin_ic_power(kk, ps, amp) /
                      (box * box * box));
  uint64_t m = ((uint64_t)ix * n + iy) * nh + iz;
  double g1, g2;
  draw_pair(key, m, &g1, &g2);
  *re = scale * g1 / sqrt(2.0);
  *im = scale * g2 / sqrt(2.0);
}

static int fill(int n, double box, uint64_t seed, const pin_spectrum* ps,
                double* out64, float* out32) {
  if (n < 2 || (n & 1) || box <= 0.0 || ps == NULL || (out64 == NULL && out32 == NULL))
    return -1;
  const int nh = n / 2 + 1;
  const double amp = pin_ic_amplitude(ps);
  const uint64_t key = pin_ic_splitmix64(seed);
#pragma omp parallel for schedule(static)
  for (int ix = 0; ix < n; ++ix) {
    for (int iy = 0; iy < n; ++iy) {
      for (int iz = 0; iz < nh; ++iz) {
        size_t m = ((size_t)ix * n + iy) * nh + iz;
        double re = 0.0, im = 0.0;
        if (!(ix == 0 && iy == 0 && iz == 0)) {
          if (iz == 0 || iz == n / 2) {
            int jx = (n - ix) % n, jy = (n - iy) % n;
            size_t mm = ((size_t)jx * n + jy) * nh + iz;
            if (mm == m) {
              mode_value(n, box, key, ps, amp, ix, iy, iz, &re, &im);
              re *= sqrt(2.0);
              im = 0.0;
            } else if (mm < m) {
              mode_value(n, box, key, ps, amp, jx, jy, iz, &re, &im);
              im = -im;
            } else {
              mode_value(n, box, key, ps, amp, ix, iy, iz, &re, &im);
            }
          } else {
            mode_value(n, box, key, ps, amp, ix, iy, iz, &re, &im);
          }
        }
        if (out64) { out64[2 * m] = re; out64[2 * m + 1] = im; }
        if (out32) { out32[2 * m] = (float)re; out32[2 * m + 1] = (float)im; }
      }
    }
  }
  return 0;
}

int pin_ic_delta_k(int n, double box, uint64_t seed, const pin_spectrum* ps, double* out) {
  return fill(n, box, seed, ps, out, NULL);
}

int pin_ic_delta_k_f32(int n, double box, uint64_t seed, const pin_spectrum* ps, float* out) {
  return fill(n, box, seed, ps, NULL, out);
}
