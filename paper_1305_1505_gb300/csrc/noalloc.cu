// pin_collapse_times_noalloc: the collapse-time loop for small grids with no
// device allocation at all (declared in include/pin.h).
//
// Who needs it: callers that cannot allocate device memory at call time.  A
// serving process that has already handed the device's memory to its own pool
// has none left for a per-call cudaMalloc; code that runs inside an allocator
// hook must not re-enter the allocator; and a latency-critical caller cannot
// accept cudaFree's implicit device-wide synchronisation.  Such callers pass
// device inputs and outputs, and the workspace (the half-spectra between the
// passes, the per-radius filter tables, the FP64-redo counters) lives in one
// file-scope device array below, sized for grids up to PIN_NOALLOC_MAX_N.
//
// That array exists once per device and stays allocated on every GPU that
// loads this library until the process exits.  All calls share it and it keeps
// the previous call's contents, so every call rewrites what it reads (tables,
// spectra including their pad columns) and zeroes its counters; two calls
// whose work overlaps on the GPU (different streams, or different host
// threads) race on it and must be serialised by the caller.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "kernels.cuh"
#include "pin.h"

namespace {

constexpr int kMaxN = PIN_NOALLOC_MAX_N;
constexpr int kMaxNhp = (kMaxN / 2 + 2) & ~1;
constexpr size_t kSpecElems = (size_t)kMaxN * kMaxN * kMaxNhp;  // one padded half-spectrum
constexpr size_t kSpecBytes = kSpecElems * sizeof(float2);
constexpr size_t kMultBytes = (size_t)64 * 3 * kMaxN * sizeof(float);
constexpr size_t kTwBytes = (size_t)kMaxN * sizeof(float2);
constexpr size_t kOffPhi0 = 0;
constexpr size_t kOffU = kOffPhi0 + kSpecBytes;
constexpr size_t kOffV = kOffU + 3 * kSpecBytes;
constexpr size_t kOffMult = kOffV + 6 * kSpecBytes;
constexpr size_t kOffTw = kOffMult + kMultBytes;
constexpr size_t kRedoCap = (size_t)kMaxN * kMaxN * kMaxN / 64;
constexpr size_t kOffCnt = kOffTw + kTwBytes;
constexpr size_t kOffRedoCount = kOffCnt + 4 * sizeof(unsigned long long);
constexpr size_t kOffErr = kOffRedoCount + 16;  // cleared with the counters
constexpr size_t kOffRedo = (kOffErr + sizeof(int) + 255) & ~(size_t)255;
constexpr size_t kScratchBytes = (kOffRedo + kRedoCap * sizeof(pin::RedoEntry) + 255) & ~(size_t)255;

// The whole workspace of this entry point (about 11.3 MB for N <= 64).  In host
// code this name is only a stand-in for the symbol, never a device address:
// the address comes from cudaGetSymbolAddress at set-up.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
unsigned char* g_scratch_ptr[kMaxDevices] = {};

struct Radii {
  double r[64];
};

// Per-radius axis multipliers {W, kW, k^2 W}/n (kW zero on the Nyquist index)
// and the level-2 twiddles w_n^{p k1} in [k1][p] order, computed on the device
// so that nothing is staged through host memory.
__global__ void k_noalloc_tables(Radii radii, int nscales, int n, double box, int E, int P,
                                 float* mult, float2* tw) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int total = nscales * n;
  if (tid < total) {
    const int s = tid / n, i = tid % n;
    const int si = i < n / 2 ? i : i - n;
    const double k = 2.0 * M_PI * si / box;
    const double R = radii.r[s];
    const double w = exp(-0.5 * k * k * R * R) / n;
    float* m = mult + (size_t)s * 3 * n;
    m[i] = (float)w;
    m[n + i] = (i == n / 2) ? 0.0f : (float)(k * w);
    m[2 * n + i] = (float)(k * k * w);
  }
  if (tid < E * P) {
    const int k1 = tid / P, q = tid % P;
    double sn, cs;
    sincospi(2.0 * (double)((q * k1) % n) / n, &sn, &cs);
    tw[tid] = make_float2((float)cs, (float)sn);
  }
}

// Phi0(k) = delta(k) / k^2 into the padded layout (pad modes and k = 0 zero).
__global__ void k_noalloc_phi0(const void* src, int dtype, int n, int nhp, double box, float2* phi0) {
  const int nh = n / 2 + 1;
  const size_t total = (size_t)n * n * nhp;
  const double kf = 2.0 * M_PI / box;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    const int iz = (int)(i % nhp);
    const size_t row = i / nhp;
    const int iy = (int)(row % n), ix = (int)(row / n);
    float2 out = make_float2(0.f, 0.f);
    if (iz < nh) {
      const size_t j = row * nh + iz;
      float2 d;
      if (dtype == PIN_C64) {
        d = static_cast<const float2*>(src)[j];
      } else {
        const double2 dd = static_cast<const double2*>(src)[j];
        d = make_float2((float)dd.x, (float)dd.y);
      }
      const double sx = ix < n / 2 ? ix : ix - n, sy = iy < n / 2 ? iy : iy - n;
      const double sz = iz < n / 2 ? iz : -(n / 2);
      const double k2 = kf * kf * (sx * sx + sy * sy + sz * sz);
      if (k2 > 0.0) {
        const float inv = (float)(1.0 / k2);
        out = make_float2(d.x * inv, d.y * inv);
      }
    }
    phi0[i] = out;
  }
}

double noalloc_dcorr() {
  const double delta_c = 3.0 / 20.0 * std::pow(12.0 * M_PI, 2.0 / 3.0);
  double x = 2.0;  // root of x/3 + x^2/21 + 23 x^3/1701 = 1 by Newton
  for (int i = 0; i < 60; ++i) {
    const double f = x / 3.0 + x * x / 21.0 + 23.0 * x * x * x / 1701.0 - 1.0;
    const double d = 1.0 / 3.0 + 2.0 * x / 21.0 + 69.0 * x * x / 1701.0;
    const double nx = x - f / d;
    if (nx == x) break;
    x = nx;
  }
  return 1.0 / delta_c - 1.0 / x;
}

// Once per device, with that device current: the scratch address, the
// constant twiddle tables and the kernels' shared-memory limits.
pin_status noalloc_setup(int dev, unsigned char** out) {
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (!g_scratch_ptr[dev]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || ptr == nullptr) return PIN_ECUDA;
    if (pin::upload_constant_twiddles() != cudaSuccess) return PIN_ECUDA;
    for (int n : {8, 16, 32, 48, 64})
      if (pin::prepare_kernels(n) != cudaSuccess) return PIN_ECUDA;
    g_scratch_ptr[dev] = static_cast<unsigned char*>(ptr);
  }
  *out = g_scratch_ptr[dev];
  return PIN_OK;
}

}  // namespace

extern "C" pin_status pin_collapse_times_noalloc(const void* delta_k, int dtype, int n, double box,
                                                 int nscales, const double* radii, int correction,
                                                 float* F_max, int32_t* scale_idx, void* stream) {
  if (!delta_k || !radii || !F_max || !scale_idx) return PIN_EINVAL;
  if (n > kMaxN || n < 8 || !pin::size_supported(n)) return PIN_EINVAL;  // beyond the static workspace
  if (dtype != PIN_C64 && dtype != PIN_C128) return PIN_EINVAL;
  if (nscales < 1 || nscales > 64 || !(box > 0.0) || !std::isfinite(box)) return PIN_EINVAL;
  if (correction != PIN_CORR_NONE && correction != PIN_CORR_SPHERE) return PIN_EINVAL;
  Radii rr{};
  for (int s = 0; s < nscales; ++s) {
    if (!(radii[s] >= 0.0) || !std::isfinite(radii[s])) return PIN_EINVAL;
    rr.r[s] = radii[s];
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PIN_ECUDA;
  unsigned char* base = nullptr;
  pin_status st = noalloc_setup(dev, &base);
  if (st != PIN_OK) return st;

  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  const pin::PassShape sh = pin::pass_shape(n);
  const int nhp = (n / 2 + 2) & ~1;
  const size_t spec = (size_t)n * n * nhp;
  float2* phi0 = reinterpret_cast<float2*>(base + kOffPhi0);
  float2* U = reinterpret_cast<float2*>(base + kOffU);
  float2* V = reinterpret_cast<float2*>(base + kOffV);
  float* mult = reinterpret_cast<float*>(base + kOffMult);
  float2* tw = reinterpret_cast<float2*>(base + kOffTw);
  unsigned long long* cnt = reinterpret_cast<unsigned long long*>(base + kOffCnt);
  unsigned* redo_count = reinterpret_cast<unsigned*>(base + kOffRedoCount);
  int* err = reinterpret_cast<int*>(base + kOffErr);
  CUtensorMap tm_x, tm_y;
  const int tc = pin::pass_shape(n).tc;  // the default tile width
  if (pin::make_tmap_x(&tm_x, phi0, n, n, nhp, 1, tc) != cudaSuccess ||
      pin::make_tmap_y(&tm_y, U, n, n, nhp, spec, 1, tc) != cudaSuccess)
    return PIN_ECUDA;
  pin::RedoEntry* redo_list = reinterpret_cast<pin::RedoEntry*>(base + kOffRedo);
  const double dcorr = noalloc_dcorr();
  const size_t n3 = (size_t)n * n * n;

  const int tthreads = 128;
  const int tblocks = (nscales * n + tthreads - 1) / tthreads;
  k_noalloc_tables<<<tblocks, tthreads, 0, cs>>>(rr, nscales, n, box, sh.E, sh.P, mult, tw);
  k_noalloc_phi0<<<(unsigned)((spec + 255) / 256), 256, 0, cs>>>(delta_k, dtype, n, nhp, box, phi0);
  if (cudaGetLastError() != cudaSuccess) return PIN_ECUDA;
  if (cudaMemsetAsync(cnt, 0, 4 * sizeof(unsigned long long) + 32, cs) != cudaSuccess ||
      cudaMemsetAsync(F_max, 0, n3 * sizeof(float), cs) != cudaSuccess ||
      cudaMemsetAsync(scale_idx, 0xFF, n3 * sizeof(int32_t), cs) != cudaSuccess)
    return PIN_ECUDA;

  static const int vout[6] = {0, 3, 4, 1, 2, 5};
  static const int sel[6] = {2, 1, 1, 0, 0, 0};
  static const int ym[6] = {0, 1, 0, 2, 0, 1};
  static const int zm[6] = {0, 0, 1, 0, 2, 1};
  for (int s = 0; s < nscales; ++s) {
    const float* m = mult + (size_t)s * 3 * n;
    pin::ArgsX ax{};
    ax.tm = tm_x;
    ax.src = phi0;
    for (int f = 0; f < 3; ++f) { ax.dst[f] = U + f * spec; ax.xm[f] = f; }
    ax.nout = 3;
    ax.ny = n;
    ax.mult = m;
    ax.tw = tw;
    ax.nhp = nhp;
    ax.batch = 1;
    ax.err = err;
    pin::ArgsY ay{};
    ay.tm = tm_y;
    for (int f = 0; f < 3; ++f) ay.src[f] = U + f * spec;
    for (int o = 0; o < 6; ++o) {
      ay.dst[o] = V + vout[o] * spec;
      ay.sel[o] = sel[o];
      ay.ym[o] = ym[o];
      ay.zm[o] = zm[o];
      ay.muli[o] = 0;
    }
    ay.nout = 6;
    ay.nx = n;
    ay.nz = n;
    ay.mult = m;
    ay.mult_z = m;  // cubic grid: one table serves every axis
    ay.tw = tw;
    ay.nhp = nhp;
    ay.batch = 1;
    ay.err = err;
    pin::ArgsZ az{};
    for (int f = 0; f < 6; ++f) az.src[f] = V + f * spec;
    az.nfields = 6;
    az.nlines = n * n;
    az.npart = n * n * n;
    az.lam_out = reinterpret_cast<float*>(U);
    az.tw = tw;
    az.nhp = nhp;
    az.fmax = F_max;
    az.idx = scale_idx;
    az.scale = s;
    az.correction = correction;
    az.dcorr_d = dcorr;
    az.dcorr_f = (float)dcorr;
    az.tau_eig = 2e-4f;
    az.tau_root = 1e-3f;
    az.counters = cnt;
    az.redo_list = redo_list;
    az.redo_count = redo_count;
    az.redo_cap = (unsigned)kRedoCap;
    if (pin::launch_x(n, tc, ax, cs) != cudaSuccess || pin::launch_y(n, tc, ay, cs) != cudaSuccess ||
        cudaMemsetAsync(redo_count, 0, sizeof(unsigned), cs) != cudaSuccess ||
        pin::launch_z(n, az, false, cs) != cudaSuccess ||
        (!pin::z_fuses_roots(n) && pin::launch_roots(az, cs) != cudaSuccess) ||
        pin::launch_redo(az, cs) != cudaSuccess)
      return PIN_ECUDA;
  }
  return PIN_OK;
}
