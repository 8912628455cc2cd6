// C-ABI of the collapse-time path (declared in include/pin.h).
//
// A plan owns the device workspace of one grid size and radius list:
//   phi0            Phi0(k) = delta(k) / k^2, half-spectrum, padded stride nhp
//   U[3], V[6]      outputs of the x and y passes
//   fmax, idx       running maximum of F and its radius index (Sec. 2.1.1)
//   mult            per-radius axis multipliers {W, kW, k^2 W} / N
// pin_collapse_times replays one CUDA graph holding the whole radius loop.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "kernels.cuh"
#include "pin.h"
#include "pin_ic.h"

using namespace pin;

struct pin_plan_s {
  int nx = 0, ny = 0, nz = 0, nhp = 0, nscales = 0, correction = 1, precision = 0;
  int batch = 1;          // realisations sharing the grid and radii
  bool velocities = false; // keep the smoothed displacement at R_max (v_max)
  double box = 0.0;
  std::vector<double> radii;
  std::vector<int> order;  // radius indices by ascending radius (ties: index), the loop's order
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  PassShape shape_x{}, shape_y{}, shape_z{};  // line transforms along x, y, z
  size_t spec_elems = 0;  // complex elements of one padded half-spectrum
  size_t field_elems = 0; // batch * spec_elems: one field of every realisation
  float2* phi0 = nullptr;
  float2* U = nullptr;    // 3 spectra
  float2* V = nullptr;    // 6 spectra (9 with velocities)
  float* psi = nullptr;   // [3][npart] displacement of the current radius (velocities)
  float* vstate = nullptr;  // [3][npart] displacement at R_max (velocities)
  float* fmax = nullptr;
  int* idx = nullptr;
  float* mult = nullptr;  // kMaxScales + 1 sets of 3 x n; set kMaxScales has R = 0
  float2* tw = nullptr;
  unsigned long long* counters = nullptr;  // [0] eig redo, [1] root redo, [2] queue overflow
  RedoEntry* redo_list = nullptr;          // FP64 redo queue, reused by every radius
  unsigned* redo_count = nullptr;
  unsigned redo_cap = 0;
  int* err = nullptr;                      // set by a pass whose bounded TMA wait gave up
  long long wait_cycles = 0;               // TMA wait budget of the x/y passes (0: default)
  CUtensorMap tm_x{}, tm_y{};              // Phi0 -> x pass, U[3] -> y pass
  int tc_x = 0, tc_y = 0;                  // tile widths (columns per block) of the x and y passes
  int vx = 0, vy = 0;                      // radix schedules of the x and y line transforms
  bool ic_set = false;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  // graphs captured for other radius lists (pin_set_radii), keyed by the order
  // their loop runs the radius indices in (the tables are read from device
  // memory, so a graph serves every list with that order); cleared with the
  // current graph
  std::map<std::vector<int>, std::pair<cudaGraph_t, cudaGraphExec_t>> graph_cache;
  uint64_t calls = 0;
  double dcorr = 0.0;
  bool profile = false;             // graph carries per-pass event records
  std::vector<cudaEvent_t> events;  // 7 per radius: x begin/end, y begin/end, z begin/end, redo end
  // radius schedule (pin_set_schedule): 0 serial; 1 the z pass and redo of
  // radius s on a second stream while the x pass of s + 1 runs; 2 also the y
  // pass of s + 1, into a second set of V spectra
  int sched = 0;
  cudaStream_t s_xy = nullptr, s_z = nullptr;  // high / low priority streams of the overlapped schedule
  float2* V2 = nullptr;                        // second V buffer (schedule 2)
  // PIN_FP64 plans: FP64 half-spectrum, one full complex cube, the tensor,
  // F_max in FP64 (fp64.cu)
  double2* d64 = nullptr;
  double2* w64 = nullptr;
  double* h64 = nullptr;
  double* fmax64 = nullptr;
  std::vector<cudaEvent_t> cap_ev;             // fork/join events of the overlapped capture
  std::string last_error;
  size_t tw_off[3] = {0, 0, 0};  // per-axis twiddle tables within tw (x, y, z)
  size_t n3() const { return (size_t)nx * ny * nz; }
  // multiplier set ms: [3][nx] for x, then [3][ny] for y, then [3][nz] for z
  size_t mult_set() const { return 3 * (size_t)(nx + ny + nz); }
  const float* mx(int ms) const { return mult + ms * mult_set(); }
  const float* my(int ms) const { return mx(ms) + 3 * (size_t)nx; }
  const float* mz(int ms) const { return my(ms) + 3 * (size_t)ny; }
  const float2* twx() const { return tw + tw_off[0]; }
  const float2* twy() const { return tw + tw_off[1]; }
  const float2* twz() const { return tw + tw_off[2]; }
  // cubic cells: side of an axis with nax points (exactly box along x)
  double len(int nax) const { return nax == nx ? box : box * nax / nx; }
};

namespace pin {

// kz stride of the half-spectra: n/2 + 1 modes rounded up to a multiple of 4
// complex values, so that every row starts on a 32-byte sector (column tiles
// of the y pass then write whole sectors; rows also meet the 16-byte TMA
// stride rule)
int padded_half(int n) { return (n / 2 + 1 + 3) & ~3; }

static double delta_c_value() { return 3.0 / 20.0 * std::pow(12.0 * M_PI, 2.0 / 3.0); }

// Uncorrected spherical collapse root: x/3 + x^2/21 + 23 x^3/1701 = 1, Newton
// from x = 2 (the function is increasing and convex on x > 0).
static double x3_value() {
  double x = 2.0;
  for (int i = 0; i < 60; ++i) {
    double f = x / 3.0 + x * x / 21.0 + 23.0 * x * x * x / 1701.0 - 1.0;
    double d = 1.0 / 3.0 + 2.0 * x / 21.0 + 69.0 * x * x / 1701.0;
    double nx = x - f / d;
    if (nx == x) break;
    x = nx;
  }
  return x;
}

double correction_dcorr() { return 1.0 / delta_c_value() - 1.0 / x3_value(); }

// Per-axis multipliers for one radius: {W, k W, k^2 W} / n with
// W = exp(-k^2 R^2 / 2), k = 2 pi s / L; k W is zero on the Nyquist index.
void fill_mult(float* out, int n, double box, double radius) {
  for (int i = 0; i < n; ++i) {
    const int s = i < n / 2 ? i : i - n;
    const double k = 2.0 * M_PI * s / box;
    const double w = std::exp(-0.5 * k * k * radius * radius) / n;
    out[0 * n + i] = (float)w;
    out[1 * n + i] = (i == n / 2) ? 0.0f : (float)(k * w);
    out[2 * n + i] = (float)(k * k * w);
  }
}

// Twiddles of one axis: w_n^{p k1} in [k1][p] order; for a three-level line
// (P = P1 P2) then w_P^{p1 k2a} in [k2a][p1] order.
void fill_twiddles(float2* t, int n, const PassShape& sh) {
  const int E = sh.E, P = sh.P, P1 = sh.P1, P2 = sh.P2;
  for (int k1 = 0; k1 < E; ++k1)
    for (int q = 0; q < P; ++q) {
      const double ang = 2.0 * M_PI * (double)((long)q * k1 % n) / n;
      t[(size_t)k1 * P + q] = make_float2((float)std::cos(ang), (float)std::sin(ang));
    }
  if (P2 > 1)
    for (int k2a = 0; k2a < P2; ++k2a)
      for (int q1 = 0; q1 < P1; ++q1) {
        const double ang = 2.0 * M_PI * (double)(q1 * k2a % P) / P;
        t[(size_t)n + k2a * P1 + q1] = make_float2((float)std::cos(ang), (float)std::sin(ang));
      }
}

// Phi0(k) = delta(k) / k^2 into the padded layout (pad modes and k = 0
// zero).  Cubic cells: the side along x is `box`, L_y = box ny / nx,
// L_z = box nz / nx.
__global__ void k_load_phi0(const void* src, int dtype, int nx, int ny, int nz, int nhp, double box, int batch,
                            float2* phi0) {
  const int nh = nz / 2 + 1;
  const size_t total = (size_t)nx * ny * nhp * batch;
  const double kfx = 2.0 * M_PI / box, kfy = 2.0 * M_PI / (ny == nx ? box : box * ny / nx),
               kfz = 2.0 * M_PI / (nz == nx ? box : box * nz / nx);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    const int iz = (int)(i % nhp);
    const size_t r = i / nhp;
    const int iy = (int)(r % ny), ix = (int)((r / ny) % nx);  // r runs over realisations too
    float2 out = make_float2(0.f, 0.f);
    if (iz < nh) {
      const size_t j = r * nh + iz;
      float2 d;
      if (dtype == PIN_C64) {
        d = reinterpret_cast<const float2*>(src)[j];
      } else {
        const double2 dd = reinterpret_cast<const double2*>(src)[j];
        d = make_float2((float)dd.x, (float)dd.y);
      }
      const double sx = ix < nx / 2 ? ix : ix - nx, sy = iy < ny / 2 ? iy : iy - ny;
      const double sz = iz < nz / 2 ? iz : -(nz / 2);
      const double kx = kfx * sx, ky = kfy * sy, kz = kfz * sz;
      const double k2 = kx * kx + ky * ky + kz * kz;
      if (k2 > 0.0) {
        const float inv = (float)(1.0 / k2);
        out = make_float2(d.x * inv, d.y * inv);
      }
    }
    phi0[i] = out;
  }
}

// Plain copy by a kernel (16-byte words when both ends and the size allow,
// else 4-byte ones): used to write results into page-locked host memory
// through its device mapping.
__global__ void k_copy_out(const void* src, void* dst, size_t bytes) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  const size_t i0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if ((((uintptr_t)src | (uintptr_t)dst | bytes) & 15) == 0) {
    const uint4* s = static_cast<const uint4*>(src);
    uint4* d = static_cast<uint4*>(dst);
    for (size_t i = i0; i < bytes / 16; i += stride) d[i] = s[i];
  } else {
    const uint32_t* s = static_cast<const uint32_t*>(src);
    uint32_t* d = static_cast<uint32_t*>(dst);
    for (size_t i = i0; i < bytes / 4; i += stride) d[i] = s[i];
  }
}

// Device-to-host copy of `bytes` (a multiple of 4) on stream st: page-locked
// host memory mapped for the device is written by k_copy_out (no copy
// engine), any other host memory by cudaMemcpyAsync.
cudaError_t copy_to_host(void* host_dst, const void* dev_src, size_t bytes, cudaStream_t st) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, host_dst) == cudaSuccess && at.type == cudaMemoryTypeHost &&
      at.devicePointer != nullptr) {
    const unsigned blocks = (unsigned)std::min<size_t>((bytes / 16 + 255) / 256 + 1, 152 * 16);
    k_copy_out<<<blocks, 256, 0, st>>>(dev_src, at.devicePointer, bytes);
    return cudaGetLastError();
  }
  cudaGetLastError();  // a pageable pointer is not an error here
  return cudaMemcpyAsync(host_dst, dev_src, bytes, cudaMemcpyDeviceToHost, st);
}

cudaError_t launch_load_phi0(const void* src, int dtype, int nx, int ny, int nz, int nhp, double box, int batch,
                             float2* phi0, cudaStream_t st) {
  const size_t total = (size_t)nx * ny * nhp * batch;
  const int threads = 256;
  const unsigned blocks = (unsigned)std::min<size_t>((total + threads - 1) / threads, 152 * 64);
  k_load_phi0<<<blocks, threads, 0, st>>>(src, dtype, nx, ny, nz, nhp, box, batch, phi0);
  return cudaGetLastError();
}

}  // namespace pin

namespace {

std::mutex g_init_mu;
std::vector<int> g_tw_done;                 // per device
std::vector<std::vector<int>> g_attr_done;  // per device, per size

struct CudaFail {
  cudaError_t e;
  const char* what;
};

pin_status fail(pin_plan_t p, pin_status s, const std::string& msg) {
  if (p) p->last_error = msg;
  return s;
}

pin_status cuda_fail(pin_plan_t p, cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  return fail(p, e == cudaErrorMemoryAllocation ? PIN_ENOMEM : PIN_ECUDA, m);
}

#define PIN_CK(p, call)                                    \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return cuda_fail((p), e_, #call); \
  } while (0)

bool validate(const pin_plan_desc* d, std::string* why) {
  if (!d) { *why = "null descriptor"; return false; }
  for (int m : {d->nx, d->ny, d->nz})
    if (!size_supported(m)) { *why = "unsupported grid size " + std::to_string(m); return false; }
  if (!(d->box > 0.0) || !std::isfinite(d->box)) { *why = "box must be positive"; return false; }
  if (d->nscales < 1 || d->nscales > 64) { *why = "nscales must be in 1..64"; return false; }
  if (!d->radii) { *why = "null radii"; return false; }
  for (int s = 0; s < d->nscales; ++s)
    if (!(d->radii[s] >= 0.0) || !std::isfinite(d->radii[s])) { *why = "radii must be finite and >= 0"; return false; }
  if (d->correction != PIN_CORR_NONE && d->correction != PIN_CORR_SPHERE) { *why = "bad correction mode"; return false; }
  if (d->precision != PIN_FP32_FALLBACK64 && d->precision != PIN_FP64) { *why = "bad precision mode"; return false; }
  if (d->precision == PIN_FP64 && ((d->batch > 1) || d->velocities)) {
    *why = "PIN_FP64 needs batch 1 and no velocities";
    return false;
  }
  if (d->velocities != 0 && d->velocities != 1) { *why = "velocities must be 0 or 1"; return false; }
  const long long b = d->batch <= 0 ? 1 : d->batch;
  if (b > 4096) { *why = "batch must be in 1..4096"; return false; }
  if (b * (long long)d->nx * d->ny * d->nz >= (1ll << 31)) {
    *why = "batch * nx * ny * nz must stay below 2^31";
    return false;
  }
  return true;
}

// Host-side allocation-failure injection (pin_debug_fail_alloc): when
// g_fail_alloc >= 0, the device allocation of pin_plan with that index
// (counted from 0 over later pin_plan calls) fails as out of memory.
std::atomic<int> g_fail_alloc{-1};

cudaError_t plan_alloc(void** ptr, size_t bytes) {
  int k = g_fail_alloc.load();
  while (k >= 0) {
    if (g_fail_alloc.compare_exchange_weak(k, k - 1)) {
      if (k == 0) return cudaErrorMemoryAllocation;
      break;
    }
  }
  return cudaMalloc(ptr, bytes);
}

// FP64 redo queue capacity: 1/64 of the grid (observed rate ~2e-4), at least 64 Ki.
unsigned redo_capacity(size_t n3, int batch) {
  return (unsigned)std::max<size_t>(65536, n3 * batch / 64);
}

int batch_of(const pin_plan_desc* d) { return d->batch <= 0 ? 1 : d->batch; }

// multiplier sets of a plan: one per radius (at most 64, pin_set_radii may
// change the list), then the R = 0 set of the unsmoothed products
constexpr int kMaxScales = 64;

size_t footprint(int nx, int ny, int nz, int nscales, int batch, bool velocities, bool fp64) {
  (void)nscales;
  const size_t spec = (size_t)nx * ny * padded_half(nz) * batch;
  const size_t n3 = (size_t)nx * ny * nz * batch;
  return (fp64 ? fp64_workspace_bytes(nx, ny, nz) : 0) + spec * 8 * (velocities ? 13 : 10) + n3 * 8 +
         (velocities ? n3 * 24 : 0) +
         (size_t)(kMaxScales + 1) * 3 * (nx + ny + nz) * 4 + (size_t)(nx + ny + nz + 3 * 64) * 8 + 64 +
         (size_t)redo_capacity((size_t)nx * ny * nz, batch) * sizeof(RedoEntry) + 16 + sizeof(int);
}

pin_status ensure_device_init(pin_plan_t p) {
  std::lock_guard<std::mutex> lk(g_init_mu);
  int dev = p->device;
  if ((int)g_tw_done.size() <= dev) {
    g_tw_done.resize(dev + 1, 0);
    g_attr_done.resize(dev + 1);
  }
  if (!g_tw_done[dev]) {
    PIN_CK(p, upload_constant_twiddles());
    g_tw_done[dev] = 1;
  }
  auto& v = g_attr_done[dev];
  for (int m : {p->nx, p->ny, p->nz}) {
    if ((int)v.size() <= m) v.resize(m + 1, 0);
    if (!v[m]) {
      PIN_CK(p, prepare_kernels(m));
      v[m] = 1;
    }
  }
  return PIN_OK;
}

void drop_graph(pin_plan_t p);

void release(pin_plan_t p) {
  drop_graph(p);
  cudaFree(p->phi0);
  cudaFree(p->U);
  cudaFree(p->V);
  cudaFree(p->psi);
  cudaFree(p->vstate);
  cudaFree(p->fmax);
  cudaFree(p->idx);
  cudaFree(p->mult);
  cudaFree(p->tw);
  cudaFree(p->counters);
  cudaFree(p->redo_list);
  cudaFree(p->redo_count);
  cudaFree(p->err);
  for (cudaEvent_t e : p->events) cudaEventDestroy(e);
  p->events.clear();
  cudaFree(p->V2);
  p->V2 = nullptr;
  cudaFree(p->d64);
  cudaFree(p->w64);
  cudaFree(p->h64);
  cudaFree(p->fmax64);
  p->d64 = nullptr;
  p->w64 = nullptr;
  p->h64 = nullptr;
  p->fmax64 = nullptr;
  for (cudaEvent_t e : p->cap_ev) cudaEventDestroy(e);
  p->cap_ev.clear();
  if (p->s_xy) cudaStreamDestroy(p->s_xy);
  if (p->s_z) cudaStreamDestroy(p->s_z);
  p->s_xy = p->s_z = nullptr;
  if (p->own_stream && p->stream) cudaStreamDestroy(p->stream);
  p->graph_exec = nullptr;
  p->graph = nullptr;
}

float2* spec(pin_plan_t p, float2* base, int f) { return base + (size_t)f * p->field_elems; }

void drop_graph(pin_plan_t p) {
  if (p->graph_exec) cudaGraphExecDestroy(p->graph_exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  p->graph_exec = nullptr;
  p->graph = nullptr;
  for (auto& kv : p->graph_cache) {
    cudaGraphExecDestroy(kv.second.second);
    cudaGraphDestroy(kv.second.first);
  }
  p->graph_cache.clear();
}

// The order the radius loop runs in: ascending radius, equal radii by index.
// F_max is a maximum over radii, and the kernels break ties of F towards the
// lower radius index whatever the order, so every order gives the same
// results; smallest radii first makes most particles reach their F_max early,
// after which the z pass skips the root solve of radii that cannot beat it.
void set_order(pin_plan_t p) {
  p->order.resize(p->nscales);
  for (int s = 0; s < p->nscales; ++s) p->order[s] = s;
  std::stable_sort(p->order.begin(), p->order.end(), [&](int a, int b) { return p->radii[a] < p->radii[b]; });
}

// Multiplier sets of the plan's radii (host copy, uploaded by the caller):
// set s < nscales for radius s, set kMaxScales for R = 0.
std::vector<float> mult_table(pin_plan_t p) {
  std::vector<float> mult((size_t)(kMaxScales + 1) * p->mult_set(), 0.0f);
  for (int s = 0; s <= kMaxScales; ++s) {
    if (s < kMaxScales && s >= p->nscales) continue;
    const double R = s < p->nscales ? p->radii[s] : 0.0;
    float* m = mult.data() + (size_t)s * p->mult_set();
    fill_mult(m, p->nx, p->len(p->nx), R);
    fill_mult(m + 3 * (size_t)p->nx, p->ny, p->len(p->ny), R);
    fill_mult(m + 3 * (size_t)(p->nx + p->ny), p->nz, p->len(p->nz), R);
  }
  return mult;
}

// x pass of one radius (mult set `ms`): Phi0 -> U[0..2] with the x factors
// W, k W, k^2 W.
ArgsX radius_args_x(pin_plan_t p, int ms) {
  ArgsX ax{};
  ax.tm = p->tm_x;
  ax.src = p->phi0;
  for (int f = 0; f < 3; ++f) { ax.dst[f] = spec(p, p->U, f); ax.xm[f] = f; }
  ax.nout = 3;
  ax.ny = p->ny;
  ax.mult = p->mx(ms);
  ax.tw = p->twx();
  ax.nhp = p->nhp;
  ax.batch = p->batch;
  ax.err = p->err;
  ax.wait_cycles = p->wait_cycles;
  return ax;
}

// y pass of one radius, outputs grouped by source so that each staged tile
// serves them in a row: V[xx] <- U2; V[xy] <- U1 (k_y), V[xz] <- U1 (z: k_z);
// V[yy] <- U0 (k_y^2), V[zz] <- U0 (z: k_z^2), V[yz] <- U0 (k_y; z: k_z).
// With the velocities of a collapse call, the smoothed displacement
// psi = i k W Phi0 shares the y transforms of xz (psi_x: z factor W), zz
// (psi_z: z factor k W) and yz (psi_y: z factor W).
ArgsY radius_args_y(pin_plan_t p, int ms, bool collapse, float2* vbuf = nullptr) {
  if (!vbuf) vbuf = p->V;
  static const int vout[6] = {0, 3, 4, 1, 2, 5};
  static const int sel[6] = {2, 1, 1, 0, 0, 0};
  static const int ym[6] = {0, 1, 0, 2, 0, 1};
  static const int zm[6] = {0, 0, 1, 0, 2, 1};
  ArgsY ay{};
  ay.tm = p->tm_y;
  for (int f = 0; f < 3; ++f) ay.src[f] = spec(p, p->U, f);
  for (int o = 0; o < 6; ++o) {
    ay.dst[o] = spec(p, vbuf, vout[o]);
    ay.sel[o] = sel[o];
    ay.ym[o] = ym[o];
    ay.zm[o] = zm[o];
    ay.muli[o] = 0;
  }
  if (p->velocities && collapse) {
    ay.dst2[2] = spec(p, vbuf, 6);
    ay.zm2[2] = 0;
    ay.muli2[2] = 1;
    ay.dst2[4] = spec(p, vbuf, 8);
    ay.zm2[4] = 1;
    ay.muli2[4] = 1;
    ay.dst2[5] = spec(p, vbuf, 7);
    ay.zm2[5] = 0;
    ay.muli2[5] = 1;
  }
  ay.nout = 6;
  ay.nx = p->nx;
  ay.nz = p->nz;
  ay.mult = p->my(ms);
  ay.mult_z = p->mz(ms);
  ay.tw = p->twy();
  ay.nhp = p->nhp;
  ay.batch = p->batch;
  ay.err = p->err;
  ay.wait_cycles = p->wait_cycles;
  return ay;
}

// Where the passes of one radius of the collapse loop run: the x and y passes
// on xs, the z pass and the FP64 redo on zs, the y outputs in vbuf; the y pass
// first waits for y_wait (if set), y_done is recorded after it (and zs waits
// for it), z_done after the redo.  The serial schedule is xs = zs = the
// plan's stream, vbuf = V, no events.
struct RadiusSched {
  cudaStream_t xs, zs;
  float2* vbuf;
  cudaEvent_t y_wait, y_done, z_done;
};

// Filter-and-transform passes of one radius (mult set `ms`), ending in the
// collapse update (dump and source null), a dump of the six real components,
// or the 2LPT source field S of every particle (source, batch 1).
pin_status enqueue_radius(pin_plan_t p, int ms, int scale, float* const* dump, float* source = nullptr,
                          const RadiusSched* sched = nullptr) {
  const bool collapse = dump == nullptr && source == nullptr;
  const RadiusSched rs = sched ? *sched : RadiusSched{p->stream, p->stream, p->V, nullptr, nullptr, nullptr};
  const bool rec = p->profile && collapse && !p->events.empty();
  auto mark = [&](int k, cudaStream_t st) {
    return rec ? cudaEventRecordWithFlags(p->events[7 * scale + k], st, cudaEventRecordExternal) : cudaSuccess;
  };
  PIN_CK(p, mark(0, rs.xs));
  const ArgsX ax = radius_args_x(p, ms);
  PIN_CK(p, launch_x(p->nx, p->tc_x, p->vx, ax, rs.xs));
  PIN_CK(p, mark(1, rs.xs));
  if (rs.y_wait) PIN_CK(p, cudaStreamWaitEvent(rs.xs, rs.y_wait, 0));

  PIN_CK(p, mark(2, rs.xs));
  const ArgsY ay = radius_args_y(p, ms, collapse, rs.vbuf);
  PIN_CK(p, launch_y(p->ny, p->tc_y, p->vy, ay, rs.xs));
  PIN_CK(p, mark(3, rs.xs));
  if (rs.y_done) {
    PIN_CK(p, cudaEventRecord(rs.y_done, rs.xs));
    PIN_CK(p, cudaStreamWaitEvent(rs.zs, rs.y_done, 0));
  }

  ArgsZ az{};
  const int nf = (p->velocities && collapse) ? 9 : 6;
  for (int f = 0; f < nf; ++f) az.src[f] = spec(p, rs.vbuf, f);
  az.nfields = nf;
  az.psi_out = p->psi;
  az.vstate = (p->velocities && collapse) ? p->vstate : nullptr;
  az.nlines = p->nx * p->ny * p->batch;
  az.npart = az.nlines * p->nz;
  az.lam_out = reinterpret_cast<float*>(p->U);  // the x-pass spectra are free by now (serial schedule)
  az.tw = p->twz();
  az.nhp = p->nhp;
  az.fmax = p->fmax;
  az.idx = p->idx;
  az.scale = scale;
  az.correction = p->correction;
  az.dcorr_d = p->dcorr;
  az.dcorr_f = (float)p->dcorr;
  az.tau_eig = 2e-4f;
  az.tau_root = 1e-3f;
  az.counters = p->counters;
  az.redo_list = p->redo_list;
  az.redo_count = p->redo_count;
  az.redo_cap = p->redo_cap;
  if (dump)
    for (int f = 0; f < 6; ++f) az.out[f] = dump[f];
  if (source) {
    az.out[0] = source;
    PIN_CK(p, launch_z_source(p->nz, az, rs.zs));
    return PIN_OK;
  }
  PIN_CK(p, mark(4, rs.zs));
  if (!dump) PIN_CK(p, cudaMemsetAsync(p->redo_count, 0, sizeof(unsigned), rs.zs));
  PIN_CK(p, launch_z(p->nz, az, dump != nullptr, rs.zs));
  PIN_CK(p, mark(5, rs.zs));
  if (!dump) {
    if (!z_fuses_roots(p->nz)) PIN_CK(p, launch_roots(az, rs.zs));
    PIN_CK(p, launch_redo(az, rs.zs));
  }
  PIN_CK(p, mark(6, rs.zs));
  if (rs.z_done) PIN_CK(p, cudaEventRecord(rs.z_done, rs.zs));
  return PIN_OK;
}

pin_status enqueue_collapse(pin_plan_t p) {
  const size_t n3 = p->n3() * p->batch;
  PIN_CK(p, cudaMemsetAsync(p->fmax, 0, n3 * sizeof(float), p->stream));
  PIN_CK(p, cudaMemsetAsync(p->idx, 0xFF, n3 * sizeof(int), p->stream));
  if (p->velocities) PIN_CK(p, cudaMemsetAsync(p->vstate, 0, 3 * n3 * sizeof(float), p->stream));
  if (p->sched == 0) {
    for (int k = 0; k < p->nscales; ++k) {
      const int s = p->order[k];
      pin_status st = enqueue_radius(p, s, s, nullptr);
      if (st != PIN_OK) return st;
    }
    return PIN_OK;
  }
  // Overlapped schedule: the x and y passes of radius s + 1 run on s_xy while
  // the z pass and the redo of radius s run on s_z.  The y pass of radius s
  // overwrites the V buffer that the z pass of radius s - nbuf read, so it
  // waits for that z pass; the x pass of s writes only U, which the y pass of
  // s - 1 (earlier on s_xy) has finished reading.  Steps k run the radii in
  // the plan's order; cap_ev: [0] fork, [1 + 2 k] y_done of step k,
  // [2 + 2 k] z_done of step k.
  const int nbuf = p->sched == 2 ? 2 : 1;
  PIN_CK(p, cudaEventRecord(p->cap_ev[0], p->stream));
  PIN_CK(p, cudaStreamWaitEvent(p->s_xy, p->cap_ev[0], 0));
  PIN_CK(p, cudaStreamWaitEvent(p->s_z, p->cap_ev[0], 0));
  for (int k = 0; k < p->nscales; ++k) {
    const int s = p->order[k];
    RadiusSched rs{p->s_xy, p->s_z, (nbuf == 2 && (k & 1)) ? p->V2 : p->V,
                   k >= nbuf ? p->cap_ev[2 + 2 * (k - nbuf)] : nullptr, p->cap_ev[1 + 2 * k], p->cap_ev[2 + 2 * k]};
    pin_status st = enqueue_radius(p, s, s, nullptr, nullptr, &rs);
    if (st != PIN_OK) return st;
  }
  // join: the plan's stream continues after the last redo and the last y pass
  PIN_CK(p, cudaStreamWaitEvent(p->stream, p->cap_ev[2 + 2 * (p->nscales - 1)], 0));
  PIN_CK(p, cudaStreamWaitEvent(p->stream, p->cap_ev[1 + 2 * (p->nscales - 1)], 0));
  return PIN_OK;
}

pin_status ensure_graph(pin_plan_t p) {
  if (p->graph_exec) return PIN_OK;
  PIN_CK(p, cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeThreadLocal));
  pin_status st = enqueue_collapse(p);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(p->stream, &g);
  if (st != PIN_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) return cuda_fail(p, e, "cudaStreamEndCapture");
  p->graph = g;
  // the overlapped schedule's kernel nodes carry the priorities of their
  // capture streams (x/y passes above the z pass)
  e = cudaGraphInstantiateWithFlags(&p->graph_exec, g, p->sched ? cudaGraphInstantiateFlagUseNodePriority : 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    p->graph = nullptr;
    p->graph_exec = nullptr;
    return cuda_fail(p, e, "cudaGraphInstantiate");
  }
  return PIN_OK;
}

pin_status check_plan(pin_plan_t p) {
  if (!p) return PIN_EINVAL;
  cudaError_t e = cudaSetDevice(p->device);
  if (e != cudaSuccess) return cuda_fail(p, e, "cudaSetDevice");
  return PIN_OK;
}

// After the plan's stream has drained: a pass that gave up a bounded wait
// left its error word set.  The error is reported once, by the first check
// after it happened, and the word is cleared for the plan's later work.
pin_status check_error_word(pin_plan_t p) {
  int err = 0;
  PIN_CK(p, cudaMemcpy(&err, p->err, sizeof(int), cudaMemcpyDeviceToHost));
  if (err) {
    PIN_CK(p, cudaMemset(p->err, 0, sizeof(int)));
    return fail(p, PIN_ECUDA, "a transfer wait in the x/y pass timed out; results are invalid");
  }
  return PIN_OK;
}

pin_status finish_host(pin_plan_t p) {
  PIN_CK(p, cudaStreamSynchronize(p->stream));
  return check_error_word(p);
}

// ------------------------------------------------------------ tile tuner --
// Radix schedules and tile widths chosen by pin_autotune, per device, grid
// shape, batch and mode, shared by every plan of the process.
using TuneKey = std::tuple<int, int, int, int, int, int>;
struct TuneChoice {
  int vx, tc_x, vy, tc_y;
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneChoice> g_tune_cache;

TuneKey tune_key(pin_plan_t p) {
  return std::make_tuple(p->device, p->nx, p->ny, p->nz, p->batch, p->velocities ? 1 : 0);
}

bool tile_allowed(int n, int v, int tc) {
  int opts[2];
  const int k = xy_tile_options(n, v, opts);
  for (int i = 0; i < k; ++i)
    if (opts[i] == tc) return true;
  return false;
}

// Twiddle table of the x (axis 0) or y (axis 1) line transform for radix
// schedule v into its slot of the plan's table (the plan's stream must be
// idle).
pin_status upload_axis_twiddles(pin_plan_t p, int axis, int v) {
  const int n = axis == 0 ? p->nx : p->ny;
  const PassShape sh = pass_shape_xy(n, v);
  std::vector<float2> t((size_t)n + (sh.P2 > 1 ? sh.P : 0));
  fill_twiddles(t.data(), n, sh);
  PIN_CK(p, cudaMemcpy(p->tw + p->tw_off[axis], t.data(), t.size() * sizeof(float2), cudaMemcpyHostToDevice));
  return PIN_OK;
}

// Switches the radix schedules of the x and y passes (twiddles, shapes).
pin_status apply_radix(pin_plan_t p, int vx, int vy) {
  if (vx == p->vx && vy == p->vy) return PIN_OK;
  PIN_CK(p, cudaStreamSynchronize(p->stream));
  drop_graph(p);
  pin_status st = upload_axis_twiddles(p, 0, vx);
  if (st == PIN_OK) st = upload_axis_twiddles(p, 1, vy);
  if (st != PIN_OK) return st;
  p->vx = vx;
  p->vy = vy;
  p->shape_x = pass_shape_xy(p->nx, vx);
  p->shape_y = pass_shape_xy(p->ny, vy);
  return PIN_OK;
}

// Re-encode the plan's tensor maps for new tile widths; the captured graph
// holds the old maps and launch shapes, so it is dropped (after the stream
// drains) and captured again by the next call.
pin_status apply_tiles(pin_plan_t p, int tc_x, int tc_y) {
  CUtensorMap mx, my;
  if (make_tmap_x(&mx, p->phi0, p->nx, p->ny, p->nhp, p->batch, tc_x) != cudaSuccess ||
      make_tmap_y(&my, p->U, p->nx, p->ny, p->nhp, p->field_elems, p->batch, tc_y) != cudaSuccess)
    return fail(p, PIN_ECUDA, "tensor map encoding failed");
  PIN_CK(p, cudaStreamSynchronize(p->stream));
  drop_graph(p);
  p->tm_x = mx;
  p->tm_y = my;
  p->tc_x = tc_x;
  p->tc_y = tc_y;
  return PIN_OK;
}

// Mean device time (ms) of `reps` launches of the first radius's x or y pass
// at tile width tc with the plan's current radix schedules, after one
// untimed launch, on the plan's stream.
pin_status time_pass(pin_plan_t p, bool y_pass, int tc, int reps, float* ms) {
  ArgsX ax = radius_args_x(p, 0);
  ArgsY ay = radius_args_y(p, 0, true);
  cudaError_t e = y_pass ? make_tmap_y(&ay.tm, p->U, p->nx, p->ny, p->nhp, p->field_elems, p->batch, tc)
                         : make_tmap_x(&ax.tm, p->phi0, p->nx, p->ny, p->nhp, p->batch, tc);
  if (e != cudaSuccess) return fail(p, PIN_ECUDA, "tensor map encoding failed");
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  PIN_CK(p, cudaEventCreate(&e0));
  e = cudaEventCreate(&e1);
  for (int r = 0; e == cudaSuccess && r <= reps; ++r) {
    if (r == 1) e = cudaEventRecord(e0, p->stream);
    if (e == cudaSuccess)
      e = y_pass ? launch_y(p->ny, tc, p->vy, ay, p->stream) : launch_x(p->nx, tc, p->vx, ax, p->stream);
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, p->stream);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) return cuda_fail(p, e, "timing a pass");
  *ms = t / reps;
  return check_error_word(p);
}

}  // namespace

extern "C" {

size_t pin_footprint_bytes(const pin_plan_desc* d) {
  std::string why;
  if (!validate(d, &why)) return 0;
  return footprint(d->nx, d->ny, d->nz, d->nscales, batch_of(d), d->velocities != 0, d->precision == PIN_FP64);
}

pin_status pin_plan(pin_plan_t* out, const pin_plan_desc* d) {
  if (!out) return PIN_EINVAL;
  *out = nullptr;
  std::string why;
  if (!validate(d, &why)) return PIN_EINVAL;
  pin_plan_s* p = new (std::nothrow) pin_plan_s();
  if (!p) return PIN_ENOMEM;
  p->nx = d->nx;
  p->ny = d->ny;
  p->nz = d->nz;
  p->nhp = padded_half(p->nz);
  p->box = d->box;
  p->nscales = d->nscales;
  p->radii.assign(d->radii, d->radii + d->nscales);
  set_order(p);
  p->correction = d->correction;
  p->precision = d->precision;
  p->batch = batch_of(d);
  p->velocities = d->velocities != 0;
  p->shape_x = pass_shape_xy(p->nx, 0);
  p->shape_y = pass_shape_xy(p->ny, 0);
  p->shape_z = pass_shape(p->nz);
  p->spec_elems = (size_t)p->nx * p->ny * p->nhp;
  p->field_elems = p->spec_elems * p->batch;
  p->dcorr = correction_dcorr();
  p->redo_cap = redo_capacity(p->n3(), p->batch);
  auto bail = [&](pin_status s) {
    release(p);
    delete p;
    return s;
  };
  if (cudaGetDevice(&p->device) != cudaSuccess) return bail(PIN_ECUDA);
  if (ensure_device_init(p) != PIN_OK) return bail(PIN_ECUDA);
  if (d->stream) {
    p->stream = (cudaStream_t)d->stream;
  } else {
    if (cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking) != cudaSuccess) return bail(PIN_ECUDA);
    p->own_stream = true;
  }
  const size_t n3 = p->n3() * p->batch;
  const size_t mult_elems = (size_t)(kMaxScales + 1) * p->mult_set();
  // twiddle tables of the three axes, back to back
  const PassShape* shapes[3] = {&p->shape_x, &p->shape_y, &p->shape_z};
  const int ns[3] = {p->nx, p->ny, p->nz};
  size_t tw_elems = 0;
  for (int a = 0; a < 3; ++a) {
    p->tw_off[a] = tw_elems;
    // the x and y slots hold the table of either radix schedule (at most
    // n + 64 entries: a three-level line has P <= 64 threads)
    tw_elems += (size_t)ns[a] + (a < 2 ? 64 : (shapes[a]->P2 > 1 ? shapes[a]->P : 0));
  }
  auto A = [](auto** ptr, size_t bytes) { return plan_alloc(reinterpret_cast<void**>(ptr), bytes); };
  if (A(&p->phi0, p->field_elems * 8) != cudaSuccess || A(&p->U, 3 * p->field_elems * 8) != cudaSuccess ||
      A(&p->V, (p->velocities ? 9 : 6) * p->field_elems * 8) != cudaSuccess ||
      (p->velocities && (A(&p->psi, 3 * n3 * 4) != cudaSuccess || A(&p->vstate, 3 * n3 * 4) != cudaSuccess)) ||
      A(&p->fmax, n3 * 4) != cudaSuccess || A(&p->idx, n3 * 4) != cudaSuccess ||
      A(&p->mult, mult_elems * 4) != cudaSuccess || A(&p->tw, tw_elems * 8) != cudaSuccess ||
      A(&p->counters, 3 * sizeof(unsigned long long)) != cudaSuccess ||
      A(&p->redo_list, (size_t)p->redo_cap * sizeof(RedoEntry)) != cudaSuccess ||
      A(&p->redo_count, sizeof(unsigned)) != cudaSuccess || A(&p->err, sizeof(int)) != cudaSuccess ||
      (p->precision == PIN_FP64 &&
       (A(&p->d64, (size_t)p->nx * p->ny * (p->nz / 2 + 1) * 16) != cudaSuccess ||
        A(&p->w64, n3 * 16) != cudaSuccess || A(&p->h64, 6 * n3 * 8) != cudaSuccess ||
        A(&p->fmax64, n3 * 8) != cudaSuccess))) {
    cudaGetLastError();
    return bail(PIN_ENOMEM);
  }
  const std::vector<float> mult = mult_table(p);
  std::vector<float2> tw(tw_elems);
  for (int a = 0; a < 3; ++a) fill_twiddles(tw.data() + p->tw_off[a], ns[a], *shapes[a]);
  if (cudaMemcpy(p->mult, mult.data(), mult_elems * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(p->tw, tw.data(), tw.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(p->counters, 0, 3 * sizeof(unsigned long long)) != cudaSuccess ||
      cudaMemset(p->err, 0, sizeof(int)) != cudaSuccess)
    return bail(PIN_ECUDA);
  p->tc_x = p->shape_x.tc;
  p->tc_y = p->shape_y.tc;
  if (make_tmap_x(&p->tm_x, p->phi0, p->nx, p->ny, p->nhp, p->batch, p->tc_x) != cudaSuccess ||
      make_tmap_y(&p->tm_y, p->U, p->nx, p->ny, p->nhp, p->field_elems, p->batch, p->tc_y) != cudaSuccess)
    return bail(PIN_ECUDA);
  *out = p;
  return PIN_OK;
}

pin_status pin_set_ic(pin_plan_t p, const void* delta_k, int dtype, int on_device) {
  pin_status st = check_plan(p);
  if (st != PIN_OK) return st;
  if (!delta_k) return fail(p, PIN_EINVAL, "null delta_k");
  if (dtype != PIN_C64 && dtype != PIN_C128) return fail(p, PIN_EINVAL, "dtype must be PIN_C64 or PIN_C128");
  const size_t nh = (size_t)p->nz / 2 + 1;
  const size_t bytes = (size_t)p->nx * p->ny * nh * (dtype == PIN_C64 ? 8 : 16) * p->batch;
  const void* src = delta_k;
  if (!on_device) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, delta_k) == cudaSuccess && at.type == cudaMemoryTypeHost &&
        at.devicePointer != nullptr) {
      // page-locked host memory, mapped for the device: the Phi0 kernel reads
      // it in place (one pass over the host data, no staging copy; its many
      // loads in flight keep the host link busy where a copy engine waits
      // on address translation)
      src = at.devicePointer;
    } else {
      cudaGetLastError();  // a pageable pointer is not an error here
      // stage through the V workspace (6 spectra >= one C128 half-spectrum)
      PIN_CK(p, cudaMemcpyAsync(p->V, delta_k, bytes, cudaMemcpyHostToDevice, p->stream));
      src = p->V;
    }
  }
  PIN_CK(p, launch_load_phi0(src, dtype, p->nx, p->ny, p->nz, p->nhp, p->box, p->batch, p->phi0, p->stream));
  if (p->d64) PIN_CK(p, fp64_load(src, dtype, p->nx, p->ny, p->nz, p->d64, p->stream));
  if (!on_device) PIN_CK(p, cudaStreamSynchronize(p->stream));
  p->ic_set = true;
  return PIN_OK;
}

pin_status pin_set_ic_seed(pin_plan_t p, uint64_t seed, const pin_spectrum* ps) {
  pin_status st = check_plan(p);
  if (st != PIN_OK) return st;
  if (!ps) return fail(p, PIN_EINVAL, "null spectrum");
  if (p->nx != p->ny || p->ny != p->nz) return fail(p, PIN_EINVAL, "pin_set_ic_seed needs a cubic grid");
  if (!(ps->gamma > 0.0) || !std::isfinite(ps->ns) || !(ps->sigma8 > 0.0))
    return fail(p, PIN_EINVAL, "bad spectrum parameters");
  const double amp = pin_ic_amplitude(ps);
  std::vector<uint64_t> keys(p->batch);
  for (int b = 0; b < p->batch; ++b) keys[b] = pin_ic_splitmix64(seed + (uint64_t)b);
  // stage: the keys after the generated half-spectra in the V workspace (>= 6 spectra)
  const size_t half = (size_t)p->nx * p->nx * (p->nx / 2 + 1) * p->batch;
  float2* field = p->V;
  uint64_t* keys_dev = reinterpret_cast<uint64_t*>(p->V + half + 1);
  PIN_CK(p, cudaMemcpyAsync(keys_dev, keys.data(), keys.size() * sizeof(uint64_t), cudaMemcpyHostToDevice,
                            p->stream));
  PIN_CK(p, generate_ic(p->nx, p->box, keys_dev, p->batch, amp, ps->ns, ps->gamma, field, p->stream));
  PIN_CK(p, launch_load_phi0(field, PIN_C64, p->nx, p->ny, p->nz, p->nhp, p->box, p->batch, p->phi0, p->stream));
  if (p->d64) PIN_CK(p, fp64_load(field, PIN_C64, p->nx, p->ny, p->nz, p->d64, p->stream));
  PIN_CK(p, cudaStreamSynchronize(p->stream));  // the host key vector goes out of scope
  p->ic_set = true;
  return PIN_OK;
}

// The FP64 radius loop of a PIN_FP64 plan into fmax64 / idx, and its FP32
// copy into fmax (kept for the calls that read F_max, e.g. the fragment order).
pin_status run_fp64(pin_plan_t p) {
  const size_t n3 = p->n3();
  PIN_CK(p, fp64_collapse(p->d64, p->nx, p->ny, p->nz, p->box, p->nscales, p->radii.data(), p->correction, p->dcorr,
                          p->w64, p->h64, p->fmax64, p->idx, p->stream));
  PIN_CK(p, fp64_cast(p->fmax64, n3, p->fmax, p->stream));
  return PIN_OK;
}

pin_status pin_collapse_times(pin_plan_t p, float* F_max, int32_t* scale_idx, int on_device) {
  pin_status st = check_plan(p);
  if (st != PIN_OK) return st;
  if (!F_max || !scale_idx) return fail(p, PIN_EINVAL, "null output");
  if (!p->ic_set) return fail(p, PIN_ESTATE, "pin_set_ic has not been called");
  if (p->precision == PIN_FP64) {
    st = run_fp64(p);
  } else {
    st = ensure_graph(p);
    if (st == PIN_OK) PIN_CK(p, cudaGraphLaunch(p->graph_exec, p->stream));
  }
  if (st != PIN_OK) return st;
  const size_t n3 = p->n3() * p->batch;
  if (on_device) {
    PIN_CK(p, cudaMemcpyAsync(F_max, p->fmax, n3 * 4, cudaMemcpyDeviceToDevice, p->stream));
    PIN_CK(p, cudaMemcpyAsync(scale_idx, p->idx, n3 * 4, cudaMemcpyDeviceToDevice, p->stream));
  } else {
    PIN_CK(p, copy_to_host(F_max, p->fmax, n3 * 4, p->stream));
    PIN_CK(p, copy_to_host(scale_idx, p->idx, n3 * 4, p->stream));
  }
  p->calls++;
  if (!on_device) return finish_host(p);
  return PIN_OK;
}

pin_status pin_collapse_times_f64(pin_plan_t p, double* F_max, int32_t* scale_idx, int on_device) {
  pin_status st = check_plan(p);
  if (st != PIN_OK) return st;
  if (!F_max || !scale_idx) return fail(p, PIN_EINVAL, "null output");
  if (p->precision != PIN_FP64) return fail(p, PIN_EINVAL, "pin_collapse_times_f64 needs a PIN_FP64 plan");
  if (!p->ic_set) return fail(p, PIN_ESTATE, "pin_set_ic has not been called");
  st = run_fp64(p);
  if (st != PIN_OK) return st;
  const size_t n3 = p->n3();
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  PIN_CK(p, cudaMemcpyAsync(F_max, p->fmax64, n3 * 8, kind, p->stream));
  PIN_CK(p, cudaMemcpyAsync(scale_idx, p->idx, n3 * 4, kind, p->stream));
  p->calls++;
  if (!on_device) return finish_host(p);
  return PIN_OK;
}

pin_status pin_velocities(pin_plan_t p, float* psi_max, int on_device) {
  pin_status st = check_plan(p);
  if (st != PIN_OK) return st;
  if (!psi_max) return fail(p, PIN_EINVAL, "null output");
  if (!p->velocities) return fail(p, PIN_EINVAL, "the plan was created without velocities");
  if (p->calls == 0) return fail(p, PIN_ESTATE, "pin_collapse_times has not been called");
  const size_t n3 = p->n3() * p->batch;
  PIN_CK(p, cudaMemcpyAsync(psi_max, p->vstate, 3 * n3 * 4,
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, p->stream));
  if (!on_device) return finish_host(p);
  return PIN_OK;
}

pin_status pin_fragment_order(pin_plan_t p, int32_t* order, uint8_t* n_before, int on_device) {
  pin_status st = check_plan(p);
  if (st != PIN_OK) return st;
  if (!order && !n_before) return fail(p, PIN_EINVAL, "both outputs are null");
  if (p->batch != 1) return fail(p, PIN_EINVAL, "pin_fragment_order needs a plan with batch 1");
  if (p->calls == 0) return fail(p, PIN_ESTATE, "pin_collapse_times has not been called");
  const long n3 = (long)p->n3();
  // the y-pass spectra are free once the radius loop is done: sort scratch,
  // and (for host outputs) the device copies of the results after it
  const size_t need = fragment_scratch_bytes(n3);
  const size_t have = (size_t)(p->velocities ? 9 : 6) * p->field_elems * sizeof(float2);
  const size_t tail = (need + 255) & ~(size_t)255;
  if (tail + (size_t)n3 > have) return fail(p, PIN_ECUDA, "fragment scratch does not fit the plan's workspace");
  char* scratch = reinterpret_cast<char*>(p->V);
  int32_t* order_dev = order;
  uint8_t* nb_dev = n_before;
  if (!on_device) {
    // the last radix pass reads keys and values A and writes only values:
    // the second value array is free for the order
    if (order) order_dev = reinterpret_cast<int32_t*>(scratch + (size_t)3 * n3 * 4);
    if (n_before) nb_dev = reinterpret_cast<uint8_t*>(scratch + tail);
  }
  PIN_CK(p, fragment_order(p->fmax, p->nx, p->ny, p->nz, scratch, order_dev, nb_dev, p->stream));
  if (!on_device) {
    if (order) PIN_CK(p, cudaMemcpyAsync(order, order_dev, (size_t)n3 * 4, cudaMemcpyDeviceToHost, p->stream));
    if (n_before) PIN_CK(p, cudaMemcpyAsync(n_before, nb_dev, (size_t)n3, cudaMemcpyDeviceToHost, p->stream));
    return finish_host(p);
  }
  return PIN_OK;
}

pin_status pin_hessian(pin_plan_t p, int scale, float* out6, int on_device) {
  pin_status st = check_plan(p);
  if (st != PIN_OK) return st;
  if (!out6) return fail(p, PIN_EINVAL, "null output");
  if (scale < 0 || scale >= p->nscales) return fail(p, PIN_EINVAL, "scale index out of range");
  if (p->batch != 1) return fail(p, PIN_EINVAL, "pin_hessian needs a plan with batch 1");
  if (!p->ic_set) return fail(p, PIN_ESTATE, "pin_set_ic has not been called");
  const size_t n3 = p->n3();
  float* dev = out6;
  if (!on_device) PIN_CK(p, cudaMallocAsync((void**)&dev, 6 * n3 * 4, p->stream));
  float* outs[6];
  for (int f = 0; f < 6; ++f) outs[f] = dev + (size_t)f * n3;
  st = enqueue_radius(p, scale, scale, outs);
  if (st == PIN_OK && !on_device) {
    cudaError_t e = cudaMemcpyAsync(out6, dev, 6 * n3 * 4, cudaMemcpyDeviceToHost, p->stream);
    if (e != cudaSuccess) st = cuda_fail(p, e, "cudaMemcpyAsync");
  }
  if (!on_device) {
    cudaFreeAsync(dev, p->stream);
    if (st == PIN_OK) st = finish_host(p);
  }
  return st;
}

// The three displacement passes psi = IDFT(i k Phi) of a potential spectrum
// Phi (padded half-spectrum, R = 0: no smoothing), through the spectra a0, a1
// (x-pass outputs, stored back to back) and b0..b2 (y-pass outputs), into
// out = [3][N^3].
static cudaError_t enqueue_gradient(pin_plan_t p, float2* phi, float2* a0, float2* b0, float* out) {
  const size_t n3 = p->n3();
  const int r0 = kMaxScales;  // the R = 0 multiplier set
  ArgsX ax{};
  cudaError_t e = make_tmap_x(&ax.tm, phi, p->nx, p->ny, p->nhp, 1, p->tc_x);
  if (e != cudaSuccess) return e;
  ax.src = phi;
  ax.dst[0] = a0;
  ax.dst[1] = a0 + p->field_elems;
  ax.xm[0] = 0;
  ax.xm[1] = 1;
  ax.nout = 2;
  ax.ny = p->ny;
  ax.mult = p->mx(r0);
  ax.tw = p->twx();
  ax.nhp = p->nhp;
  ax.batch = 1;
  ax.err = p->err;
  ax.wait_cycles = p->wait_cycles;
  e = launch_x(p->nx, p->tc_x, p->vx, ax, p->stream);
  if (e != cudaSuccess) return e;
  // psi_x <- a1 (k_x), psi_y <- a0 (k_y), psi_z <- a0 (z: k_z); all times i
  ArgsY ay{};
  e = make_tmap_y(&ay.tm, a0, p->nx, p->ny, p->nhp, p->field_elems, 1, p->tc_y);
  if (e != cudaSuccess) return e;
  ay.src[0] = a0;
  ay.src[1] = a0 + p->field_elems;
  ay.src[2] = a0 + 2 * p->field_elems;
  const int sel[3] = {1, 0, 0}, ym[3] = {0, 1, 0}, zm[3] = {0, 0, 1};
  for (int f = 0; f < 3; ++f) {
    ay.dst[f] = b0 + (size_t)f * p->field_elems;
    ay.sel[f] = sel[f];
    ay.ym[f] = ym[f];
    ay.zm[f] = zm[f];
    ay.muli[f] = 1;
  }
  ay.nout = 3;
  ay.nx = p->nx;
  ay.nz = p->nz;
  ay.mult = p->my(r0);
  ay.mult_z = p->mz(r0);
  ay.tw = p->twy();
  ay.nhp = p->nhp;
  ay.batch = 1;
  ay.err = p->err;
  ay.wait_cycles = p->wait_cycles;
  e = launch_y(p->ny, p->tc_y, p->vy, ay, p->stream);
  if (e != cudaSuccess) return e;
  ArgsZ az{};
  for (int f = 0; f < 3; ++f) {
    az.src[f] = b0 + (size_t)f * p->field_elems;
    az.out[f] = out + (size_t)f * n3;
  }
  az.nfields = 3;
  az.nlines = p->nx * p->ny;
  az.tw = p->twz();
  az.nhp = p->nhp;
  return launch_z(p->nz, az, true, p->stream);
}

pin_status pin_displacements(pin_plan_t p, float* psi, int on_device) {
  pin_status st = check_plan(p);
  if (st != PIN_OK) return st;
  if (!psi) return fail(p, PIN_EINVAL, "null output");
  if (p->batch != 1) return fail(p, PIN_EINVAL, "pin_displacements needs a plan with batch 1");
  if (!p->ic_set) return fail(p, PIN_ESTATE, "pin_set_ic has not been called");
  const size_t n3 = p->n3();
  float* dev = psi;
  if (!on_device) PIN_CK(p, cudaMallocAsync((void**)&dev, 3 * n3 * 4, p->stream));
  cudaError_t e = enqueue_gradient(p, p->phi0, spec(p, p->U, 0), spec(p, p->V, 0), dev);
  if (e != cudaSuccess) st = cuda_fail(p, e, "displacement passes");
  if (st == PIN_OK && !on_device) {
    e = cudaMemcpyAsync(psi, dev, 3 * n3 * 4, cudaMemcpyDeviceToHost, p->stream);
    if (e != cudaSuccess) st = cuda_fail(p, e, "cudaMemcpyAsync");
  }
  if (!on_device) {
    cudaFreeAsync(dev, p->stream);
    if (st == PIN_OK) st = finish_host(p);
  }
  return st;
}

pin_status pin_displacements_2lpt(pin_plan_t p, float* psi2, int on_device) {
  pin_status st = check_plan(p);
  if (st != PIN_OK) return st;
  if (!psi2) return fail(p, PIN_EINVAL, "null output");
  if (p->batch != 1) return fail(p, PIN_EINVAL, "pin_displacements_2lpt needs a plan with batch 1");
  if (!p->ic_set) return fail(p, PIN_ESTATE, "pin_set_ic has not been called");
  const int nx = p->nx, ny = p->ny, nz = p->nz;
  const size_t n3 = p->n3();
  float* dev = psi2;
  if (!on_device) PIN_CK(p, cudaMallocAsync((void**)&dev, 3 * n3 * 4, p->stream));
  float2* U0 = spec(p, p->U, 0);
  float2* V0 = spec(p, p->V, 0);
  float* S = reinterpret_cast<float*>(U0);  // nx ny nz floats fit in one padded spectrum
  // 1) the unsmoothed deformation tensor, reduced per particle to the source S
  st = enqueue_radius(p, kMaxScales, 0, nullptr, S);
  // 2) T = inverse-sign transform of S: z into V0, y into V1, x into V2; the
  //    R = 0 multipliers scale each y line by 1/ny, each x line by 1/nx and
  //    the y outputs by 1/nz (z factor), so T / (nx ny nz) arrives in V2
  cudaError_t e = cudaSuccess;
  if (st == PIN_OK) e = launch_fwd_z(nz, S, V0, nx * ny, p->nhp, p->twz(), p->stream);
  if (st == PIN_OK && e == cudaSuccess) {
    const int r0 = kMaxScales;
    ArgsY ay{};
    e = make_tmap_y(&ay.tm, V0, nx, ny, p->nhp, p->field_elems, 1, p->tc_y);
    ay.src[0] = V0;
    ay.src[1] = V0;
    ay.src[2] = V0;
    ay.dst[0] = spec(p, p->V, 1);
    ay.nout = 1;
    ay.nx = nx;
    ay.nz = nz;
    ay.mult = p->my(r0);
    ay.mult_z = p->mz(r0);
    ay.tw = p->twy();
    ay.nhp = p->nhp;
    ay.batch = 1;
    ay.err = p->err;
    ay.wait_cycles = p->wait_cycles;
    if (e == cudaSuccess) e = launch_y(ny, p->tc_y, p->vy, ay, p->stream);
    ArgsX ax{};
    if (e == cudaSuccess) e = make_tmap_x(&ax.tm, spec(p, p->V, 1), nx, ny, p->nhp, 1, p->tc_x);
    ax.src = spec(p, p->V, 1);
    ax.dst[0] = spec(p, p->V, 2);
    ax.nout = 1;
    ax.ny = ny;
    ax.mult = p->mx(r0);
    ax.tw = p->twx();
    ax.nhp = p->nhp;
    ax.batch = 1;
    ax.err = p->err;
    ax.wait_cycles = p->wait_cycles;
    if (e == cudaSuccess) e = launch_x(nx, p->tc_x, p->vx, ax, p->stream);
    // 3) Phi2 = (3/7) S(k) / k^2 with S(k) = conj(T) (forward transform of real S), into U0
    if (e == cudaSuccess)
      e = launch_phi2(spec(p, p->V, 2), U0, nx, ny, nz, p->nhp, p->box, (float)(3.0 / 7.0 * (double)n3),
                      p->stream);
    // 4) psi2 = IDFT(i k Phi2)
    if (e == cudaSuccess) e = enqueue_gradient(p, U0, spec(p, p->V, 0), spec(p, p->V, 3), dev);
    if (e != cudaSuccess) st = cuda_fail(p, e, "2LPT passes");
  }
  if (st == PIN_OK && !on_device) {
    e = cudaMemcpyAsync(psi2, dev, 3 * n3 * 4, cudaMemcpyDeviceToHost, p->stream);
    if (e != cudaSuccess) st = cuda_fail(p, e, "cudaMemcpyAsync");
  }
  if (!on_device) {
    cudaFreeAsync(dev, p->stream);
    if (st == PIN_OK) st = finish_host(p);
  }
  return st;
}

pin_status pin_sync(pin_plan_t p, int64_t timeout_ns) {
  pin_status st = check_plan(p);
  if (st != PIN_OK) return st;
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    cudaError_t e = cudaStreamQuery(p->stream);
    if (e == cudaSuccess) return check_error_word(p);
    if (e != cudaErrorNotReady) return cuda_fail(p, e, "cudaStreamQuery");
    if (timeout_ns >= 0) {
      const auto dt = std::chrono::duration_cast<std::chrono::nanoseconds>(
                          std::chrono::steady_clock::now() - t0).count();
      if (dt >= timeout_ns) return fail(p, PIN_ETIMEOUT, "pin_sync timed out");
    }
    std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
}

pin_status pin_get_stats(pin_plan_t p, pin_stats* out) {
  pin_status st = check_plan(p);
  if (st != PIN_OK) return st;
  if (!out) return fail(p, PIN_EINVAL, "null stats");
  unsigned long long c[3] = {0, 0, 0};
  PIN_CK(p, cudaMemcpyAsync(c, p->counters, sizeof(c), cudaMemcpyDeviceToHost, p->stream));
  PIN_CK(p, cudaStreamSynchronize(p->stream));
  out->eig_fp64_redo = c[0];
  out->root_fp64_redo = c[1];
  out->fp64_queue_overflow = c[2];
  out->collapse_calls = p->calls;
  return PIN_OK;
}

int pin_kernels_per_call(pin_plan_t p) {
  if (!p) return 0;
  return (z_fuses_roots(p->nz) ? 4 : 5) * p->nscales;  // x, y, z, [roots,] redo per radius
}

pin_status pin_profile(pin_plan_t p, int enable) {
  pin_status st = check_plan(p);
  if (st != PIN_OK) return st;
  const bool want = enable != 0;
  if (want == p->profile) return PIN_OK;
  PIN_CK(p, cudaStreamSynchronize(p->stream));
  if (want && p->events.empty()) {
    p->events.resize(7 * (size_t)kMaxScales, nullptr);
    for (auto& e : p->events) PIN_CK(p, cudaEventCreate(&e));
  }
  p->profile = want;
  drop_graph(p);  // rebuilt with (or without) the event records
  return PIN_OK;
}

pin_status pin_tile_options(int n, int* opts, int* count) {
  return pin_tile_options_radix(n, 0, opts, count);
}

pin_status pin_tile_options_radix(int n, int radix, int* opts, int* count) {
  if (!opts || !count) return PIN_EINVAL;
  const int k = xy_tile_options(n, radix, opts);
  if (k == 0) return PIN_EINVAL;
  *count = k;
  return PIN_OK;
}

int pin_radix_schedules(void) { return kRadixVariants; }

pin_status pin_radix_shape(int n, int radix, int* E, int* P1, int* P2) {
  if (!E || !P1 || !P2) return PIN_EINVAL;
  if (!size_supported(n) || radix < 0 || radix >= kRadixVariants) return PIN_EINVAL;
  const PassShape sh = pass_shape_xy(n, radix);
  *E = sh.E;
  *P1 = sh.P1;
  *P2 = sh.P2;
  return PIN_OK;
}

pin_status pin_get_radix(pin_plan_t p, int* vx, int* vy) {
  pin_status st = check_plan(p);
  if (st != PIN_OK) return st;
  if (!vx || !vy) return fail(p, PIN_EINVAL, "null output");
  *vx = p->vx;
  *vy = p->vy;
  return PIN_OK;
}

pin_status pin_set_radix(pin_plan_t p, int vx, int vy) {
  pin_status st = check_plan(p);
  if (st != PIN_OK) return st;
  if (vx < 0 || vx >= kRadixVariants || vy < 0 || vy >= kRadixVariants)
    return fail(p, PIN_EINVAL, "radix schedule must be in 0..pin_radix_schedules()-1");
  st = apply_radix(p, vx, vy);
  if (st != PIN_OK) return st;
  // keep the tile widths if the new schedules run them, else their defaults
  const int tx = tile_allowed(p->nx, vx, p->tc_x) ? p->tc_x : p->shape_x.tc;
  const int ty = tile_allowed(p->ny, vy, p->tc_y) ? p->tc_y : p->shape_y.tc;
  if (tx == p->tc_x && ty == p->tc_y) return PIN_OK;
  return apply_tiles(p, tx, ty);
}

pin_status pin_get_tiles(pin_plan_t p, int* tc_x, int* tc_y) {
  pin_status st = check_plan(p);
  if (st != PIN_OK) return st;
  if (!tc_x || !tc_y) return fail(p, PIN_EINVAL, "null output");
  *tc_x = p->tc_x;
  *tc_y = p->tc_y;
  return PIN_OK;
}

pin_status pin_set_tiles(pin_plan_t p, int tc_x, int tc_y) {
  pin_status st = check_plan(p);
  if (st != PIN_OK) return st;
  if (tc_x == 0) tc_x = p->shape_x.tc;
  if (tc_y == 0) tc_y = p->shape_y.tc;
  if (!tile_allowed(p->nx, p->vx, tc_x) || !tile_allowed(p->ny, p->vy, tc_y))
    return fail(p, PIN_EINVAL, "tile width is not one of the plan's radix schedule's options");
  if (tc_x == p->tc_x && tc_y == p->tc_y) return PIN_OK;
  return apply_tiles(p, tc_x, tc_y);
}

pin_status pin_autotune(pin_plan_t p, int reps, int flags, int* tc_x, int* tc_y) {
  pin_status st = check_plan(p);
  if (st != PIN_OK) return st;
  if (reps < 1 || reps > 1000) return fail(p, PIN_EINVAL, "reps must be in 1..1000");
  if (flags & ~PIN_TUNE_FORCE) return fail(p, PIN_EINVAL, "unknown flags");
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  PIN_CK(p, cudaStreamIsCapturing(p->stream, &cap));
  if (cap != cudaStreamCaptureStatusNone) return fail(p, PIN_ESTATE, "the plan's stream is being captured");
  const auto key = tune_key(p);
  TuneChoice best{0, 0, 0, 0};
  bool cached = false;
  if (!(flags & PIN_TUNE_FORCE)) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      best = it->second;
      cached = true;
    }
  }
  if (!cached) {
    // the passes only read Phi0 (zeros until a field is set) and write the
    // U and V workspaces; F_max, the index and v_max are untouched.  Every
    // (radix schedule, tile width) candidate of each pass is timed.
    if (!p->ic_set) PIN_CK(p, cudaMemsetAsync(p->phi0, 0, p->field_elems * sizeof(float2), p->stream));
    const int vx0 = p->vx, vy0 = p->vy;
    float best_ms[2] = {0.f, 0.f};
    bool have[2] = {false, false};
    for (int v = 0; v < kRadixVariants; ++v) {
      st = apply_radix(p, v, v);
      if (st != PIN_OK) return st;
      for (int pass = 0; pass < 2; ++pass) {
        int opts[2];
        const int k = xy_tile_options(pass ? p->ny : p->nx, v, opts);
        for (int i = 0; i < k; ++i) {
          float ms = 0.f;
          st = time_pass(p, pass == 1, opts[i], reps, &ms);
          if (st != PIN_OK) return st;
          if (!have[pass] || ms < best_ms[pass]) {
            have[pass] = true;
            best_ms[pass] = ms;
            if (pass) { best.vy = v; best.tc_y = opts[i]; }
            else { best.vx = v; best.tc_x = opts[i]; }
          }
        }
      }
    }
    st = apply_radix(p, vx0, vy0);
    if (st != PIN_OK) return st;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = best;
  }
  st = apply_radix(p, best.vx, best.vy);
  if (st != PIN_OK) return st;
  if (best.tc_x != p->tc_x || best.tc_y != p->tc_y) {
    st = apply_tiles(p, best.tc_x, best.tc_y);
    if (st != PIN_OK) return st;
  }
  if (tc_x) *tc_x = p->tc_x;
  if (tc_y) *tc_y = p->tc_y;
  return PIN_OK;
}

pin_status pin_pass_times(pin_plan_t p, double* ms4) {
  pin_status st = check_plan(p);
  if (st != PIN_OK) return st;
  if (!ms4) return fail(p, PIN_EINVAL, "null output");
  if (!p->profile || p->events.empty() || p->calls == 0) return fail(p, PIN_ESTATE, "profiling is off or nothing ran");
  PIN_CK(p, cudaStreamSynchronize(p->stream));
  ms4[0] = ms4[1] = ms4[2] = ms4[3] = 0.0;
  // events per radius: x begin/end, y begin/end, z begin/end, redo end
  static const int from[4] = {0, 2, 4, 5}, to[4] = {1, 3, 5, 6};
  for (int s = 0; s < p->nscales; ++s)
    for (int k = 0; k < 4; ++k) {
      float ms = 0.f;
      PIN_CK(p, cudaEventElapsedTime(&ms, p->events[7 * s + from[k]], p->events[7 * s + to[k]]));
      ms4[k] += ms;
    }
  return PIN_OK;
}

pin_status pin_set_radii(pin_plan_t p, int nscales, const double* radii) {
  pin_status st = check_plan(p);
  if (st != PIN_OK) return st;
  if (nscales < 1 || nscales > kMaxScales) return fail(p, PIN_EINVAL, "nscales must be in 1..64");
  if (!radii) return fail(p, PIN_EINVAL, "null radii");
  for (int s = 0; s < nscales; ++s)
    if (!(radii[s] >= 0.0) || !std::isfinite(radii[s])) return fail(p, PIN_EINVAL, "radii must be finite and >= 0");
  PIN_CK(p, cudaStreamSynchronize(p->stream));  // no work in flight reads the old tables
  const std::vector<int> old_order = p->order;
  p->nscales = nscales;
  p->radii.assign(radii, radii + nscales);
  set_order(p);
  if (p->order != old_order) {
    // keep the current graph for its order; take a kept one for the new order
    if (p->graph_exec) {
      p->graph_cache[old_order] = {p->graph, p->graph_exec};
      p->graph = nullptr;
      p->graph_exec = nullptr;
    }
    auto it = p->graph_cache.find(p->order);
    if (it != p->graph_cache.end()) {
      p->graph = it->second.first;
      p->graph_exec = it->second.second;
      p->graph_cache.erase(it);
    }
  }
  const std::vector<float> mult = mult_table(p);
  PIN_CK(p, cudaMemcpy(p->mult, mult.data(), (size_t)nscales * p->mult_set() * sizeof(float), cudaMemcpyHostToDevice));
  return PIN_OK;
}

pin_status pin_set_schedule(pin_plan_t p, int schedule) {
  pin_status st = check_plan(p);
  if (st != PIN_OK) return st;
  if (schedule < 0 || schedule > 2) return fail(p, PIN_EINVAL, "schedule must be 0, 1 or 2");
  if (schedule && !z_fuses_roots(p->nz))
    return fail(p, PIN_EINVAL, "the overlapped schedules need a z pass that computes the collapse times (nz 384, 768)");
  if (schedule == p->sched) return PIN_OK;
  PIN_CK(p, cudaStreamSynchronize(p->stream));
  if (schedule && !p->s_xy) {
    int least = 0, greatest = 0;
    PIN_CK(p, cudaDeviceGetStreamPriorityRange(&least, &greatest));
    PIN_CK(p, cudaStreamCreateWithPriority(&p->s_xy, cudaStreamNonBlocking, greatest));
    PIN_CK(p, cudaStreamCreateWithPriority(&p->s_z, cudaStreamNonBlocking, least));
    p->cap_ev.assign(1 + 2 * (size_t)kMaxScales, nullptr);
    for (auto& e : p->cap_ev) PIN_CK(p, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  }
  if (schedule == 2 && !p->V2) {
    cudaError_t e = plan_alloc(reinterpret_cast<void**>(&p->V2), (size_t)(p->velocities ? 9 : 6) * p->field_elems * 8);
    if (e != cudaSuccess) {
      p->V2 = nullptr;
      cudaGetLastError();
      return fail(p, PIN_ENOMEM, "no device memory for the second V buffer of schedule 2");
    }
  }
  if (schedule != 2 && p->V2) {
    cudaFree(p->V2);
    p->V2 = nullptr;
  }
  p->sched = schedule;
  drop_graph(p);
  return PIN_OK;
}

int pin_get_schedule(pin_plan_t p) { return p ? p->sched : -1; }

pin_status pin_set_wait_budget(pin_plan_t p, int64_t cycles) {
  pin_status st = check_plan(p);
  if (st != PIN_OK) return st;
  if (cycles < 0) return fail(p, PIN_EINVAL, "the wait budget must be >= 0 (0: the default)");
  if ((long long)cycles == p->wait_cycles) return PIN_OK;
  PIN_CK(p, cudaStreamSynchronize(p->stream));
  p->wait_cycles = (long long)cycles;
  drop_graph(p);  // the captured launches carry the old budget
  return PIN_OK;
}

void pin_debug_fail_alloc(int nth) { g_fail_alloc.store(nth < 0 ? -1 : nth); }

const char* pin_strerror(pin_status s) {
  switch (s) {
    case PIN_OK: return "ok";
    case PIN_EINVAL: return "invalid argument";
    case PIN_ENOMEM: return "out of device memory";
    case PIN_ECUDA: return "CUDA error";
    case PIN_EBUSY: return "busy";
    case PIN_ETIMEOUT: return "timed out";
    case PIN_ESTATE: return "call out of order";
    default: return "unknown status";
  }
}

const char* pin_last_error(pin_plan_t p) { return p ? p->last_error.c_str() : ""; }

void pin_destroy(pin_plan_t p) {
  if (!p) return;
  cudaSetDevice(p->device);
  if (p->stream) cudaStreamSynchronize(p->stream);
  release(p);
  delete p;
}

}  // extern "C"
