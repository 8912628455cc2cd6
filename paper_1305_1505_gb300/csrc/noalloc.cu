// pin_collapse_times_noalloc: the collapse-time loop for small grids with no
// device allocation at all, and pin_noalloc_status, which reads back what its
// last call recorded (both declared in include/pin.h).
//
// Who needs it: callers that cannot allocate device memory at call time.  A
// serving process that has already handed the device's memory to its own pool
// has none left for a per-call cudaMalloc; code that runs inside an allocator
// hook must not re-enter the allocator; and a latency-critical caller cannot
// accept cudaFree's implicit device-wide synchronisation.  Such callers pass
// device inputs and outputs, and the workspace (the half-spectra between the
// passes, the per-radius filter tables, the FP64 redo queue, its counters and
// the error word) lives in one file-scope device array below, sized for grids
// up to PIN_NOALLOC_MAX_N.
//
// That array exists once per device and stays allocated on every GPU that
// loads this library until the process exits.  All calls share it and it keeps
// the previous call's contents, so every call rewrites what it reads (tables,
// spectra including their pad columns) and zeroes its counters and error word;
// two calls whose work overlaps on the GPU (different streams, or different
// host threads) race on it and must be serialised by the caller.
//
// The tables are built on the host by the same functions as the plan path's
// (fill_mult, fill_twiddles, padded_half, the redo capacity), staged in a
// file-scope host array and copied in on the caller's stream, and the same
// kernels run with the same launch shapes, so the results equal
// pin_collapse_times bit for bit.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "kernels.cuh"
#include "pin.h"

namespace {

constexpr int kMaxN = PIN_NOALLOC_MAX_N;
constexpr int kMaxScales = 64;
constexpr int kMaxNhp = (kMaxN / 2 + 1 + 3) & ~3;  // padded_half(kMaxN)
constexpr size_t kSpecElems = (size_t)kMaxN * kMaxN * kMaxNhp;  // one padded half-spectrum
constexpr size_t kSpecBytes = kSpecElems * sizeof(float2);
constexpr size_t kMultFloats = (size_t)kMaxScales * 3 * kMaxN;
constexpr size_t kMultBytes = kMultFloats * sizeof(float);
constexpr size_t kTwBytes = (size_t)kMaxN * sizeof(float2);
// FP64 redo queue: the plan path's capacity, max(65536, N^3 / 64), which is
// 65536 entries for every N this entry point accepts
constexpr size_t kRedoCap = 65536;
static_assert((size_t)kMaxN * kMaxN * kMaxN / 64 <= kRedoCap, "redo capacity below the plan path's rule");
constexpr size_t kOffPhi0 = 0;
constexpr size_t kOffU = kOffPhi0 + kSpecBytes;
constexpr size_t kOffV = kOffU + 3 * kSpecBytes;
constexpr size_t kOffMult = kOffV + 6 * kSpecBytes;
constexpr size_t kOffTw = kOffMult + kMultBytes;
constexpr size_t kOffCnt = kOffTw + kTwBytes;                 // 3 counters
constexpr size_t kOffRedoCount = kOffCnt + 4 * sizeof(unsigned long long);
constexpr size_t kOffErr = kOffRedoCount + 16;                // cleared with the counters
constexpr size_t kStatusBytes = kOffErr + 16 - kOffCnt;      // counters .. error word
constexpr size_t kOffRedo = (kOffErr + 16 + 255) & ~(size_t)255;
constexpr size_t kScratchBytes = (kOffRedo + kRedoCap * sizeof(pin::RedoEntry) + 255) & ~(size_t)255;

// The whole device workspace of this entry point (13.9 MB for
// N <= 64).  In host code this name is only a stand-in for the symbol, never
// a device address: the address comes from cudaGetSymbolAddress at set-up.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
unsigned char* g_scratch_ptr[kMaxDevices] = {};

// Host staging of the tables (filled and copied under g_stage_mu; a copy from
// pageable host memory has consumed its source when cudaMemcpyAsync returns).
std::mutex g_stage_mu;
float g_h_mult[kMultFloats];
float2 g_h_tw[kMaxN];

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

int current_device() {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return -1;
  return dev;
}

}  // namespace

extern "C" pin_status pin_collapse_times_noalloc(const void* delta_k, int dtype, int n, double box,
                                                 int nscales, const double* radii, int correction,
                                                 float* F_max, int32_t* scale_idx, void* stream) {
  if (!delta_k || !radii || !F_max || !scale_idx) return PIN_EINVAL;
  if (n > kMaxN || n < 8 || !pin::size_supported(n)) return PIN_EINVAL;  // beyond the static workspace
  if (dtype != PIN_C64 && dtype != PIN_C128) return PIN_EINVAL;
  if (nscales < 1 || nscales > kMaxScales || !(box > 0.0) || !std::isfinite(box)) return PIN_EINVAL;
  if (correction != PIN_CORR_NONE && correction != PIN_CORR_SPHERE) return PIN_EINVAL;
  for (int s = 0; s < nscales; ++s)
    if (!(radii[s] >= 0.0) || !std::isfinite(radii[s])) return PIN_EINVAL;
  const int dev = current_device();
  if (dev < 0) return PIN_ECUDA;
  unsigned char* base = nullptr;
  pin_status st = noalloc_setup(dev, &base);
  if (st != PIN_OK) return st;

  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  const pin::PassShape sh = pin::pass_shape(n);
  const int nhp = pin::padded_half(n);
  const size_t spec = (size_t)n * n * nhp;
  float2* phi0 = reinterpret_cast<float2*>(base + kOffPhi0);
  float2* U = reinterpret_cast<float2*>(base + kOffU);
  float2* V = reinterpret_cast<float2*>(base + kOffV);
  float* mult = reinterpret_cast<float*>(base + kOffMult);
  float2* tw = reinterpret_cast<float2*>(base + kOffTw);
  unsigned long long* cnt = reinterpret_cast<unsigned long long*>(base + kOffCnt);
  unsigned* redo_count = reinterpret_cast<unsigned*>(base + kOffRedoCount);
  int* err = reinterpret_cast<int*>(base + kOffErr);
  pin::RedoEntry* redo_list = reinterpret_cast<pin::RedoEntry*>(base + kOffRedo);
  CUtensorMap tm_x, tm_y;
  const int tc = sh.tc;  // the default tile width, as a new plan runs
  if (pin::make_tmap_x(&tm_x, phi0, n, n, nhp, 1, tc) != cudaSuccess ||
      pin::make_tmap_y(&tm_y, U, n, n, nhp, spec, 1, tc) != cudaSuccess)
    return PIN_ECUDA;
  const double dcorr = pin::correction_dcorr();
  const size_t n3 = (size_t)n * n * n;
  {
    // per radius [3][n] multipliers (cubic grid: one table serves all axes)
    std::lock_guard<std::mutex> lk(g_stage_mu);
    for (int s = 0; s < nscales; ++s) pin::fill_mult(g_h_mult + (size_t)s * 3 * n, n, box, radii[s]);
    pin::fill_twiddles(g_h_tw, n, sh);
    if (cudaMemcpyAsync(mult, g_h_mult, (size_t)nscales * 3 * n * sizeof(float), cudaMemcpyHostToDevice, cs) !=
            cudaSuccess ||
        cudaMemcpyAsync(tw, g_h_tw, (size_t)n * sizeof(float2), cudaMemcpyHostToDevice, cs) != cudaSuccess)
      return PIN_ECUDA;
  }
  if (pin::launch_load_phi0(delta_k, dtype, n, n, n, nhp, box, 1, phi0, cs) != cudaSuccess) return PIN_ECUDA;
  if (cudaMemsetAsync(cnt, 0, kStatusBytes, cs) != cudaSuccess ||
      cudaMemsetAsync(F_max, 0, n3 * sizeof(float), cs) != cudaSuccess ||
      cudaMemsetAsync(scale_idx, 0xFF, n3 * sizeof(int32_t), cs) != cudaSuccess)
    return PIN_ECUDA;

  static const int vout[6] = {0, 3, 4, 1, 2, 5};
  static const int sel[6] = {2, 1, 1, 0, 0, 0};
  static const int ym[6] = {0, 1, 0, 2, 0, 1};
  static const int zm[6] = {0, 0, 1, 0, 2, 1};
  // the plan path's order: ascending radius, equal radii by index
  int order[kMaxScales];
  for (int s = 0; s < nscales; ++s) order[s] = s;
  std::stable_sort(order, order + nscales, [&](int a, int b) { return radii[a] < radii[b]; });
  for (int k = 0; k < nscales; ++k) {
    const int s = order[k];
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
    ay.mult_z = m;
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
    if (pin::launch_x(n, tc, 0, ax, cs) != cudaSuccess || pin::launch_y(n, tc, 0, ay, cs) != cudaSuccess ||
        cudaMemsetAsync(redo_count, 0, sizeof(unsigned), cs) != cudaSuccess ||
        pin::launch_z(n, az, false, cs) != cudaSuccess ||
        (!pin::z_fuses_roots(n) && pin::launch_roots(az, cs) != cudaSuccess) ||
        pin::launch_redo(az, cs) != cudaSuccess)
      return PIN_ECUDA;
  }
  return PIN_OK;
}

extern "C" pin_status pin_noalloc_status(int* wait_failed, uint64_t* counters3) {
  if (!wait_failed || !counters3) return PIN_EINVAL;
  const int dev = current_device();
  if (dev < 0) return PIN_ECUDA;
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_setup_mu);
    base = g_scratch_ptr[dev];
  }
  if (!base) return PIN_ESTATE;  // no call has run on this device
  unsigned long long c[3] = {0, 0, 0};
  int e = 0;
  if (cudaMemcpy(c, base + kOffCnt, sizeof(c), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(&e, base + kOffErr, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return PIN_ECUDA;
  *wait_failed = e != 0;
  for (int i = 0; i < 3; ++i) counters3[i] = c[i];
  return e ? PIN_ECUDA : PIN_OK;
}
