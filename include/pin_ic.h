/*
 * pin_ic.h -- seeded synthetic initial conditions for the collapse-time path.
 *
 * The paper starts every run from a realisation of a Gaussian linear density
 * field delta_l on an N^3 grid of side L, normalised so that its top-hat
 * variance at 8 Mpc/h equals sigma8^2 (Sec. 2.1.1, Eq. "deltal"), and takes the
 * generator itself from N-GenIC (Sec. 2.2).  N-GenIC's random stream is not
 * available here, so this module defines its own generator, bit-exact and
 * counter based, so that every consumer (the CUDA path, the CPU oracle used by
 * the tests, the benchmark) is fed the very same delta(k):
 *
 *   P(k)   = A k^ns T_BBKS(k/Gamma)^2          (k in h/Mpc; BBKS 1986 fit)
 *   A      : sigma8^2 / sigma^2_TH(8 Mpc/h | A=1), Simpson in ln k over
 *            [1e-5, 1e3] h/Mpc with 2^16 intervals
 *   D(k)   = sqrt(N^6 P(|k|) / L^3) (g1 + i g2) / sqrt(2)
 *   g1, g2 : Box-Muller of two uniforms drawn from splitmix64 (Steele, Lea &
 *            Flood 2014) keyed on (seed, linear mode index)
 *
 * Layout of the half-spectrum: [N][N][N/2+1] complex, row major, linear mode
 * index m = (ix*N + iy)*(N/2+1) + iz.  Signed wavenumber index
 * s(i) = i for i < N/2 and i - N otherwise (the Nyquist index maps to -N/2),
 * k = 2 pi s / L.  On the iz = 0 and iz = N/2 planes Hermitian symmetry is
 * enforced by copying the conjugate of the mirror mode (-ix, -iy) whenever the
 * mirror has the lower linear index; self-conjugate modes keep sqrt(2) times
 * their real part; the k = 0 mode is zero.  DFT convention: forward
 * D(k) = sum_q d(q) e^{-i k.q}, inverse d(q) = N^-3 sum_k D(k) e^{+i k.q}.
 *
 * This module holds none of the collapse-time arithmetic; it only produces
 * inputs.  All functions are thread-safe and deterministic (OpenMP inside).
 */
#ifndef PIN_IC_H
#define PIN_IC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  double ns;      /* primordial spectral index n (0.96 in every workload here) */
  double gamma;   /* BBKS shape parameter Gamma (0.21) */
  double sigma8;  /* top-hat rms at 8 Mpc/h (0.8) */
} pin_spectrum;

/* BBKS transfer function T(q) at q = k/Gamma (k in h/Mpc). */
double pin_ic_bbks(double q);

/* Amplitude A of P(k) = A k^ns T^2 that gives sigma(8 Mpc/h) = sigma8. */
double pin_ic_amplitude(const pin_spectrum* ps);

/* P(k) in (Mpc/h)^3 for k in h/Mpc (0 at k <= 0). */
double pin_ic_power(double k, const pin_spectrum* ps, double amplitude);

/* Fills out[2*N*N*(N/2+1)] (interleaved re, im; caller-owned host memory) with
 * the half-spectrum delta(k).  Returns 0 on success, -1 if n < 2, n odd or
 * box <= 0 or a pointer is NULL. */
int pin_ic_delta_k(int n, double box, uint64_t seed, const pin_spectrum* ps,
                   double* out);

/* Same field cast to FP32 (interleaved re, im). */
int pin_ic_delta_k_f32(int n, double box, uint64_t seed, const pin_spectrum* ps,
                       float* out);

/* splitmix64 output for state x (the published finaliser applied to
 * x + 0x9E3779B97F4A7C15); exposed so tests can check the stream. */
uint64_t pin_ic_splitmix64(uint64_t x);

#ifdef __cplusplus
}
#endif
#endif
