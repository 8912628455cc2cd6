// All-FP64 collapse-time loop (pin_plan_desc.precision = PIN_FP64): the same
// steps as the FP32 path of Sec. 2.1.1 -- filter the linear field delta(k) at
// each radius, inverse-transform the six components of the deformation tensor,
// eigenvalues and collapse time per grid point, running maximum -- in double
// precision throughout, at no attention to speed.  It is a debugging and
// checking mode of the library: every other call of a plan runs in FP32.
//
// Layout: the FP64 half-spectrum d64 [nx][ny][nz/2+1]; per component the full
// filtered cube (double2, [nx][ny][nz]) transformed in place along z, y and x
// by a mixed-radix (4, 2, 3) Stockham line transform in shared memory, one
// line per block; its real part (times 1/(nx ny nz)) into the tensor h[6][N^3];
// then per particle eig3<double> and collapse_from_eigs<double> (collapse.cuh,
// the arithmetic of the FP64 redo) and the strict running maximum.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "collapse.cuh"
#include "kernels.cuh"
#include "pin.h"

namespace pin {
namespace {

__device__ __forceinline__ double2 zadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 zsub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 zmuli(double2 a) { return make_double2(-a.y, a.x); }

// delta(k) in the caller's precision -> FP64 half-spectrum
__global__ void k_load64(const void* src, int dtype, size_t count, double2* out) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
    if (dtype == PIN_C64) {
      const float2 v = static_cast<const float2*>(src)[i];
      out[i] = make_double2(v.x, v.y);
    } else {
      out[i] = static_cast<const double2*>(src)[i];
    }
  }
}

// T_c(k) = (k_i k_j / k^2) W(kR) delta(k) on the full cube of modes (the
// half-spectrum's mirror modes as conjugates; k = 0 and, for i != j, every mode
// with k_i or k_j on the Nyquist index set to zero).  Cubic cells: the side
// along x is `box`, L_y = box ny / nx, L_z = box nz / nx.
__global__ void k_fill64(const double2* half, int nx, int ny, int nz, double box, double radius, int ci, int cj,
                         double2* full) {
  const int nh = nz / 2 + 1;
  const size_t n3 = (size_t)nx * ny * nz;
  const int ns[3] = {nx, ny, nz};
  const double kf[3] = {2.0 * M_PI / box, 2.0 * M_PI / (ny == nx ? box : box * ny / nx),
                        2.0 * M_PI / (nz == nx ? box : box * nz / nx)};
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n3; q += (size_t)gridDim.x * blockDim.x) {
    const int iz = (int)(q % nz), iy = (int)((q / nz) % ny), ix = (int)(q / ((size_t)nz * ny));
    const bool mirrored = iz > nz / 2;
    const size_t src = mirrored ? ((size_t)((nx - ix) % nx) * ny + (ny - iy) % ny) * nh + (nz - iz)
                                : ((size_t)ix * ny + iy) * nh + iz;
    double2 d = half[src];
    if (mirrored) d.y = -d.y;
    const int s[3] = {ix < nx / 2 ? ix : ix - nx, iy < ny / 2 ? iy : iy - ny, iz < nz / 2 ? iz : iz - nz};
    const double k[3] = {kf[0] * s[0], kf[1] * s[1], kf[2] * s[2]};
    const double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
    double2 t = make_double2(0.0, 0.0);
    const bool nyq = ci != cj && (s[ci] == -ns[ci] / 2 || s[cj] == -ns[cj] / 2);
    if (k2 > 0.0 && !nyq) {
      const double m = k[ci] * k[cj] / k2 * exp(-0.5 * k2 * radius * radius);
      t = make_double2(m * d.x, m * d.y);
    }
    full[q] = t;
  }
}

// In-place inverse transforms X[k] = sum_j x[j] exp(+2 pi i j k / n) of nlines
// lines of n points (n = 2^a 3^b), line l starting at
// (l / inner) outer_stride + (l % inner) inner_stride with elements elem_stride
// apart.  Stockham autosort, radix 4, then 2, then 3: at a stage of radix r
// with span Ns, butterfly j takes x[j + t n/r] (t < r), multiplies by
// exp(2 pi i t k / (Ns r)) with k = j mod Ns, applies the length-r DFT and
// writes element (j / Ns) Ns r + k + t Ns; the spans multiply to n.
__global__ void k_fft64(double2* data, int n, long long nlines, long long inner, long long inner_stride,
                        long long outer_stride, long long elem_stride) {
  extern __shared__ double2 zs[];
  double2* a = zs;
  double2* b = zs + n;
  for (long long l = blockIdx.x; l < nlines; l += gridDim.x) {
    double2* line = data + (l / inner) * outer_stride + (l % inner) * inner_stride;
    for (int i = threadIdx.x; i < n; i += blockDim.x) a[i] = line[(long long)i * elem_stride];
    __syncthreads();
    double2* in = a;
    double2* out = b;
    int rest = n, Ns = 1;
    while (rest > 1) {
      const int r = (rest % 4 == 0) ? 4 : (rest % 2 == 0 ? 2 : 3);
      const int m = n / r;
      for (int j = threadIdx.x; j < m; j += blockDim.x) {
        const int k = j % Ns;
        double2 v[4];
        for (int t = 0; t < r; ++t) {
          v[t] = in[j + t * m];
          if (t && k) {
            double sn, cs;
            sincospi(2.0 * (double)(t * k) / (double)(Ns * r), &sn, &cs);
            v[t] = zmul(v[t], make_double2(cs, sn));
          }
        }
        if (r == 2) {
          const double2 u0 = v[0], u1 = v[1];
          v[0] = zadd(u0, u1);
          v[1] = zsub(u0, u1);
        } else if (r == 4) {
          const double2 s02 = zadd(v[0], v[2]), d02 = zsub(v[0], v[2]);
          const double2 s13 = zadd(v[1], v[3]), d13 = zmuli(zsub(v[1], v[3]));
          v[0] = zadd(s02, s13);
          v[1] = zadd(d02, d13);
          v[2] = zsub(s02, s13);
          v[3] = zsub(d02, d13);
        } else {
          // exp(2 pi i / 3) = -1/2 + i sqrt(3)/2
          const double h = 0.86602540378443864676;
          const double2 s = zadd(v[1], v[2]), d = zsub(v[1], v[2]);
          const double2 mm = make_double2(v[0].x - 0.5 * s.x, v[0].y - 0.5 * s.y);
          v[0] = zadd(v[0], s);
          v[1] = make_double2(mm.x - h * d.y, mm.y + h * d.x);
          v[2] = make_double2(mm.x + h * d.y, mm.y - h * d.x);
        }
        const int base = (j / Ns) * Ns * r + k;
        for (int t = 0; t < r; ++t) out[base + t * Ns] = v[t];
      }
      __syncthreads();
      double2* tmp = in;
      in = out;
      out = tmp;
      Ns *= r;
      rest /= r;
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) line[(long long)i * elem_stride] = in[i];
    __syncthreads();
  }
}

__global__ void k_extract64(const double2* full, double scale, size_t n3, double* h) {
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n3; q += (size_t)gridDim.x * blockDim.x)
    h[q] = full[q].x * scale;
}

// eigenvalues, collapse time and the strict running maximum of every particle
__global__ void k_collapse64(const double* h6, size_t n3, int scale, int correction, double dcorr, double* fmax,
                             int* idx) {
  const CollapseConsts<double> cc{dcorr, correction};
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n3; q += (size_t)gridDim.x * blockDim.x) {
    double h[6], lam[3], kap;
    for (int c = 0; c < 6; ++c) h[c] = h6[c * n3 + q];
    eig3<double>(h, lam);
    const double F = collapse_from_eigs<double>(lam, cc, kap);
    if (F > fmax[q]) {
      fmax[q] = F;
      idx[q] = scale;
    }
  }
}

__global__ void k_fill_state64(size_t n3, double* fmax, int* idx) {
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n3; q += (size_t)gridDim.x * blockDim.x) {
    fmax[q] = 0.0;
    idx[q] = -1;
  }
}

__global__ void k_cast64(const double* in, size_t n3, float* out) {
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n3; q += (size_t)gridDim.x * blockDim.x)
    out[q] = (float)in[q];
}

unsigned grid_for(size_t count) { return (unsigned)std::min<size_t>((count + 255) / 256, 152 * 32); }

cudaError_t lines(double2* w, int n, long long nlines, long long inner, long long inner_stride, long long outer_stride,
                  long long elem_stride, cudaStream_t st) {
  const unsigned g = (unsigned)std::min<long long>(nlines, 152 * 64);
  k_fft64<<<g, 128, 2 * (size_t)n * sizeof(double2), st>>>(w, n, nlines, inner, inner_stride, outer_stride,
                                                            elem_stride);
  return cudaGetLastError();
}

}  // namespace

size_t fp64_workspace_bytes(int nx, int ny, int nz) {
  const size_t n3 = (size_t)nx * ny * nz, half = (size_t)nx * ny * (nz / 2 + 1);
  return half * 16 + n3 * 16 + 6 * n3 * 8 + n3 * 8;
}

cudaError_t fp64_load(const void* src, int dtype, int nx, int ny, int nz, double2* d64, cudaStream_t st) {
  const size_t count = (size_t)nx * ny * (nz / 2 + 1);
  k_load64<<<grid_for(count), 256, 0, st>>>(src, dtype, count, d64);
  return cudaGetLastError();
}

cudaError_t fp64_collapse(const double2* d64, int nx, int ny, int nz, double box, int nscales, const double* radii,
                          int correction, double dcorr, double2* work, double* h6, double* fmax, int* idx,
                          cudaStream_t st) {
  static const int ci[6] = {0, 1, 2, 0, 0, 1}, cj[6] = {0, 1, 2, 1, 2, 2};
  const size_t n3 = (size_t)nx * ny * nz;
  const double norm = 1.0 / (double)n3;
  k_fill_state64<<<grid_for(n3), 256, 0, st>>>(n3, fmax, idx);
  cudaError_t e = cudaGetLastError();
  for (int s = 0; s < nscales && e == cudaSuccess; ++s) {
    for (int c = 0; c < 6 && e == cudaSuccess; ++c) {
      k_fill64<<<grid_for(n3), 256, 0, st>>>(d64, nx, ny, nz, box, radii[s], ci[c], cj[c], work);
      e = cudaGetLastError();
      // z lines (contiguous), y lines (stride nz), x lines (stride ny nz)
      if (e == cudaSuccess) e = lines(work, nz, (long long)nx * ny, (long long)nx * ny, nz, 0, 1, st);
      if (e == cudaSuccess) e = lines(work, ny, (long long)nx * nz, nz, 1, (long long)ny * nz, nz, st);
      if (e == cudaSuccess) e = lines(work, nx, (long long)ny * nz, (long long)ny * nz, 1, 0, (long long)ny * nz, st);
      if (e == cudaSuccess) {
        k_extract64<<<grid_for(n3), 256, 0, st>>>(work, norm, n3, h6 + c * n3);
        e = cudaGetLastError();
      }
    }
    if (e == cudaSuccess) {
      k_collapse64<<<grid_for(n3), 256, 0, st>>>(h6, n3, s, correction, dcorr, fmax, idx);
      e = cudaGetLastError();
    }
  }
  return e;
}

cudaError_t fp64_cast(const double* in, size_t n3, float* out, cudaStream_t st) {
  k_cast64<<<grid_for(n3), 256, 0, st>>>(in, n3, out);
  return cudaGetLastError();
}

}  // namespace pin
