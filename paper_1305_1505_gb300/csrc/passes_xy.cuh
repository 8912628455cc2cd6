// The x and y passes of the collapse-time loop (Sec. 2.1.1): the filter
// factors of one axis fused into the inverse DFT along that axis, over column
// tiles staged in shared memory by the tensor memory accelerator.  Templated
// on the line length N, the tile width TC and the radix schedule V of the
// line transform (fft.cuh), and included by the two translation units that
// instantiate schedule 0 (kernels.cu) and schedule 1 (kernels_v1.cu).
#pragma once
#include <algorithm>
#include <cstdint>

#include "fft.cuh"
#include "kernels.cuh"

namespace pin {

// ------------------------------------------------------ TMA + mbarrier --
// Source tiles of the x and y passes are brought into shared memory by the
// tensor memory accelerator (cp.async.bulk.tensor), completing on an mbarrier.
// Every wait is bounded (the pass's wait budget, by default 2^31 SM clocks,
// about a second); a block that gives up waits once more, with the full
// default budget, for its copies in flight, reports through the pass's error
// word and returns.

__device__ __forceinline__ uint32_t smem_u32(const void* ptr) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(ptr));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_test_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
constexpr long long kWaitDefault = 1ll << 31;  // SM clocks, about a second at 2 GHz
// try_wait may suspend the thread for a while before it reports "not yet", so
// budgets below kWaitPoll clocks poll with the non-blocking test_wait instead.
constexpr long long kWaitPoll = 1ll << 16;
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, long long budget) {
  const long long t0 = clock64();
  if (budget < kWaitPoll) {
    while (!mbar_test_wait(bar, parity))
      if (clock64() - t0 > budget) return false;
    return true;
  }
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > budget) return false;
  return true;
}
// Block-uniform wait: true when the staged tile has landed for every thread.
// budget <= 0 selects the default.  On a timeout the block waits once more,
// with the default budget, for its copies in flight (so that no block exits
// with a transfer pending), records the error and the caller returns.
__device__ __forceinline__ bool stage_ready(uint32_t bar, uint32_t parity, int* err, long long budget) {
  const bool ok = mbar_wait_bounded(bar, parity, budget > 0 ? budget : kWaitDefault);
  if (__syncthreads_and(ok)) return true;
  mbar_wait_bounded(bar, parity, kWaitDefault);
  if (threadIdx.x == 0) atomicExch(err, 1);
  return false;
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* tm, int c0, int c1,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(dst), "l"(reinterpret_cast<uint64_t>(tm)), "r"(c0), "r"(c1), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* tm, int c0, int c1, uint32_t src) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];"
               ::"l"(reinterpret_cast<uint64_t>(tm)), "r"(c0), "r"(c1), "r"(src)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* tm, int c0, int c1, int c2,
                                            int c3, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];"
      ::"r"(dst), "l"(reinterpret_cast<uint64_t>(tm)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
      : "memory");
}

// Staged-tile geometry of a line length: kBoxes boxes of kRows rows (a box
// dimension is at most 256).
template <int N> struct Stage {
  static constexpr int kBoxes = (N + 255) / 256;
  static constexpr int kRows = N / kBoxes;
};

// Resident blocks per SM the register budget is sized for (shared memory
// already limits the long-line passes to one or two blocks per SM).
#ifndef PIN_XY_MINB
#define PIN_XY_MINB 1
#endif
// Outputs of the x pass, and of the y pass in single-store mode, go out by
// TMA bulk tensor stores of the output tile (written into the exchange
// buffer in tile order) instead of per-thread stores: the warps leave the
// global store queue to the copy engine (x 1.80 -> 1.62 ms, y 3.58 -> 3.36
// ms per radius at 768^3).  0 selects the per-thread stores.
#ifndef PIN_X_TMASTORE
#define PIN_X_TMASTORE 1
#endif
#ifndef PIN_Y_TMASTORE
#define PIN_Y_TMASTORE 1
#endif
#ifndef PIN_Z_MINB
#define PIN_Z_MINB 2
#endif
// Independent particles per iteration of the collapse loop.
#ifndef PIN_Z_ILP
#define PIN_Z_ILP 2
#endif
// Three-level lines hold half the registers per thread: the z pass is sized
// for more resident blocks (one line per block, 96 threads, nine blocks per
// SM at 72 registers: measured against four 192-thread blocks at 80
// registers, 768^3 z pass 5.21 -> 4.90 ms per radius); with the velocity
// fields (five transforms per line, 160 threads) four blocks.
#ifndef PIN_Z_MINB3
#define PIN_Z_MINB3 9
#endif
#ifndef PIN_Z_MINB3V
#define PIN_Z_MINB3V 4
#endif
template <int N, int TC = 16, int V = 0> struct MinBlocks {
  // three-level x/y blocks (TC columns x P threads) are sized for 512
  // resident threads per SM
  static constexpr int xy =
      Shape<N, V>::P2 > 1 ? 512 / (TC * Shape<N, V>::P) : (N >= 384 ? PIN_XY_MINB : 1);
  static constexpr int z = Shape<N>::P2 > 1 ? PIN_Z_MINB3 : (N >= 384 ? PIN_Z_MINB : 1);
  static constexpr int zv = Shape<N>::P2 > 1 ? PIN_Z_MINB3V : (N >= 384 ? PIN_Z_MINB : 1);
};

// ---------------------------------------------------------------- x pass --
// Lines along x: column index col in [0, N*nhp) enumerates (ky, kz); element
// (kx, col) sits at kx*N*nhp + col, so a row of TC columns is contiguous.  A
// persistent block walks column tiles; the staged Phi0 tile serves all
// outputs, and the next tile is requested as soon as the last output has read
// the current one into registers.  Each output tile leaves by TMA stores
// (PIN_X_TMASTORE; columns past the last are clipped by the map).
template <int N, int TC, int V>
__global__ void __launch_bounds__(TC* Shape<N, V>::P, MinBlocks<N, TC, V>::xy)
    k_pass_x(const __grid_constant__ ArgsX a) {
  constexpr int E = Shape<N, V>::E, P = Shape<N, V>::P, NTW = Shape<N, V>::kTw;
  using L = XLayoutCols<E, P, TC, Shape<N, V>::P1>;
  using G = Stage<N>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  // staged tile [N][TC]; TMA destinations start on a 128-byte boundary
  float2* s_st = reinterpret_cast<float2*>(smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127));
  float2* s_x = s_st + N * TC;
  float2* s_tw = s_x + L::kSize;
  float* s_m = reinterpret_cast<float*>(s_tw + NTW);  // [3][N] multipliers
  __shared__ __align__(8) unsigned long long s_bar;
  __shared__ float2* s_dst[3];
  __shared__ int s_xm[3];
  const int tid = threadIdx.x, c = tid % TC, p = tid / TC;
  const uint32_t bar = smem_u32(&s_bar);
  for (int i = tid; i < NTW; i += TC * P) s_tw[i] = a.tw[i];
  for (int i = tid; i < 3 * N; i += TC * P) s_m[i] = a.mult[i];
  if (tid < 3) {
    s_dst[tid] = a.dst[tid];
    s_xm[tid] = a.xm[tid];
  }
  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_init_fence();
  }
  __syncthreads();
  const int ncols = a.ny * a.nhp;
  const int tpr = (ncols + TC - 1) / TC;  // tiles per realisation; the last may run past ncols
  const int ntiles = tpr * a.batch;        // realisation r owns rows [r N, r N + N)
  auto issue = [&](int tile) {
    const int r = tile / tpr, t = tile % tpr;
    mbar_expect_tx(bar, N * TC * 8);
#pragma unroll
    for (int b = 0; b < G::kBoxes; ++b)
      tma_load_2d(smem_u32(s_st + b * G::kRows * TC), &a.tm, t * TC, r * N + b * G::kRows, bar);
  };
  if (tid == 0 && (int)blockIdx.x < ntiles) issue(blockIdx.x);
  uint32_t parity = 0;
  // TMA stores: an output tile is written into the exchange buffer in tile
  // order and stored by the copy engine; the next transform's first
  // exchange waits (in the hook) until the engine has read it
  constexpr bool kStore = PIN_X_TMASTORE != 0;
  bool pending = false;
  auto wait_store = [&] {
    if (kStore && pending) {
      if (tid == 0) bulk_wait_read();
      __syncthreads();
      pending = false;
    }
  };
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    if (!stage_ready(bar, parity, a.err, a.wait_cycles)) {
      if (kStore && tid == 0) bulk_wait_all();
      return;
    }
    parity ^= 1;
    const int col = (tile % tpr) * TC + c;
    const bool ok = col < ncols;
    const size_t rbase = (size_t)(tile / tpr) * N * ncols;
#pragma unroll 1
    for (int f = 0; f < a.nout; ++f) {
      const float* mt = s_m + s_xm[f] * N + p;
      float2 v[E];
#pragma unroll
      for (int t = 0; t < E; ++t) v[t] = cscale(s_st[(p + P * t) * TC + c], mt[P * t]);
      if (f == a.nout - 1) {
        __syncthreads();  // the tile has been read by every thread
        if (tid == 0 && tile + (int)gridDim.x < ntiles) {
          fence_proxy_async();
          issue(tile + gridDim.x);
        }
      }
      if constexpr (kStore) {
        fft_line<N, L, false, V>(v, p, c, s_x, s_tw, wait_store);
        __syncthreads();  // every thread has read its last exchange values
#pragma unroll
        for (int j = 0; j < E; ++j) s_x[fft_out_index<N, V>(p, j) * TC + c] = v[j];
        fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
          const int r = tile / tpr, t = tile % tpr;
#pragma unroll
          for (int b = 0; b < G::kBoxes; ++b)
            tma_store_2d(&a.tm_out[f], t * TC, r * N + b * G::kRows, smem_u32(s_x + b * G::kRows * TC));
          bulk_commit();
        }
        pending = true;
      } else {
        fft_line<N, L, false, V>(v, p, c, s_x, s_tw);
        float2* d = s_dst[f] + rbase + (ok ? col : 0);
#pragma unroll
        for (int j = 0; j < E; ++j)
          if (ok) d[(size_t)fft_out_index<N, V>(p, j) * ncols] = v[j];
        __syncthreads();
      }
    }
  }
  if (kStore && tid == 0) bulk_wait_all();
}

// ---------------------------------------------------------------- y pass --
// Lines along y: a tile is TC consecutive kz of one x plane; element
// (ky, kz) of plane x sits at (x*N + ky)*nhp + kz.  Columns past nhp are
// zero-filled by the tensor map and not stored.  Without second stores each
// output tile leaves by TMA stores (PIN_Y_TMASTORE); with them (DUAL) by
// per-thread stores.
template <int N, int TC, bool DUAL, int V>
__global__ void __launch_bounds__(TC* Shape<N, V>::P, MinBlocks<N, TC, V>::xy)
    k_pass_y(const __grid_constant__ ArgsY a) {
  constexpr int E = Shape<N, V>::E, P = Shape<N, V>::P, NTW = Shape<N, V>::kTw;
  using L = XLayoutCols<E, P, TC, Shape<N, V>::P1>;
  using G = Stage<N>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float2* s_st = reinterpret_cast<float2*>(smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127));
  float2* s_x = s_st + N * TC;
  float2* s_tw = s_x + L::kSize;
  float* s_m = reinterpret_cast<float*>(s_tw + NTW);
  __shared__ __align__(8) unsigned long long s_bar;
  __shared__ float2* s_dst[kMaxFields];
  __shared__ float2* s_dst2[kMaxFields];
  __shared__ int s_sel[kMaxFields], s_ym[kMaxFields], s_zm[kMaxFields], s_mi[kMaxFields];
  __shared__ int s_zm2[kMaxFields], s_mi2[kMaxFields];
  const int tid = threadIdx.x, c = tid % TC, p = tid / TC;
  const uint32_t bar = smem_u32(&s_bar);
  for (int i = tid; i < NTW; i += TC * P) s_tw[i] = a.tw[i];
  for (int i = tid; i < 3 * N; i += TC * P) s_m[i] = a.mult[i];
  if (tid < kMaxFields) {
    s_dst[tid] = a.dst[tid];
    s_sel[tid] = a.sel[tid] < 3 ? a.sel[tid] : 0;
    s_ym[tid] = a.ym[tid];
    s_zm[tid] = a.zm[tid];
    s_mi[tid] = a.muli[tid];
    s_dst2[tid] = a.dst2[tid];
    s_zm2[tid] = a.zm2[tid];
    s_mi2[tid] = a.muli2[tid];
  }
  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_init_fence();
  }
  __syncthreads();
  const int nhp = a.nhp, nout = a.nout;
  const int ktiles = (nhp + TC - 1) / TC;
  const int ntiles = a.nx * a.batch * ktiles;  // x planes of all realisations, back to back
  auto issue = [&](int tile, int src) {
    const int x = tile / ktiles, kz0 = (tile % ktiles) * TC;
    mbar_expect_tx(bar, N * TC * 8);
#pragma unroll
    for (int b = 0; b < G::kBoxes; ++b)
      tma_load_4d(smem_u32(s_st + b * G::kRows * TC), &a.tm, kz0, b * G::kRows, x, src, bar);
  };
  if (tid == 0 && (int)blockIdx.x < ntiles) issue(blockIdx.x, s_sel[0]);
  uint32_t parity = 0;
  // TMA stores (single-store mode): as in the x pass
  constexpr bool kStore = PIN_Y_TMASTORE != 0 && !DUAL;
  bool pending = false;
  auto wait_store = [&] {
    if (kStore && pending) {
      if (tid == 0) bulk_wait_read();
      __syncthreads();
      pending = false;
    }
  };
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int x = tile / ktiles, kz = (tile % ktiles) * TC + c;
    const bool ok = kz < nhp;
    const size_t base = (size_t)x * N * nhp + (ok ? kz : 0);
#pragma unroll 1
    for (int o = 0; o < nout; ++o) {
      if (o == 0 || s_sel[o] != s_sel[o - 1]) {
        if (!stage_ready(bar, parity, a.err, a.wait_cycles)) {
          if (kStore && tid == 0) bulk_wait_all();
          return;
        }
        parity ^= 1;
      }
      const float* mt = s_m + s_ym[o] * N + p;
      float2 v[E];
#pragma unroll
      for (int t = 0; t < E; ++t) v[t] = cscale(s_st[(p + P * t) * TC + c], mt[P * t]);
      const bool last_use = (o == nout - 1) || s_sel[o + 1] != s_sel[o];
      if (last_use) {
        __syncthreads();  // the staged source has been read by every thread
        if (tid == 0) {
          if (o < nout - 1) {
            fence_proxy_async();
            issue(tile, s_sel[o + 1]);
          } else if (tile + (int)gridDim.x < ntiles) {
            fence_proxy_async();
            issue(tile + gridDim.x, s_sel[0]);
          }
        }
      }
      // z factors of this column (kz <= nz/2; pad columns carry zeros anyway),
      // requested before the transform so that their latency is hidden
      const int nz = a.nz;
      const float zf = (ok && kz <= nz / 2) ? __ldg(a.mult_z + s_zm[o] * nz + kz) : 0.f;
      float zf2 = 0.f;
      if constexpr (DUAL)
        zf2 = (ok && s_dst2[o] != nullptr && kz <= nz / 2) ? __ldg(a.mult_z + s_zm2[o] * nz + kz) : 0.f;
      if constexpr (kStore) fft_line<N, L, false, V>(v, p, c, s_x, s_tw, wait_store);
      else fft_line<N, L, false, V>(v, p, c, s_x, s_tw);
      const bool mi = s_mi[o] != 0;
      float2* d = s_dst[o] + base;
      if constexpr (DUAL) {
        // outputs with a second store: the same transform with another z
        // factor (displacement components), both stores per register slot so
        // that each slot dies after its two stores
        float2* d2 = s_dst2[o];
        const bool two = ok && d2 != nullptr;
        const bool mi2 = s_mi2[o] != 0;
        d2 = two ? d2 + base : nullptr;
#pragma unroll
        for (int j = 0; j < E; ++j) {
          const size_t off = (size_t)fft_out_index<N, V>(p, j) * nhp;
          float2 w = cscale(v[j], zf);
          if (mi) w = cmuli(w);
          if (ok) d[off] = w;
          if (two) {
            float2 w2 = cscale(v[j], zf2);
            if (mi2) w2 = cmuli(w2);
            d2[off] = w2;
          }
        }
      } else if constexpr (kStore) {
        __syncthreads();  // every thread has read its last exchange values
#pragma unroll
        for (int j = 0; j < E; ++j) {
          float2 w = cscale(v[j], zf);
          if (mi) w = cmuli(w);
          s_x[fft_out_index<N, V>(p, j) * TC + c] = w;
        }
        fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
          const int kz0 = (tile % ktiles) * TC;
#pragma unroll
          for (int b = 0; b < G::kBoxes; ++b)
            tma_store_2d(&a.tm_out[o], kz0, x * N + b * G::kRows, smem_u32(s_x + b * G::kRows * TC));
          bulk_commit();
        }
        pending = true;
        continue;
      } else {
#pragma unroll
        for (int j = 0; j < E; ++j) {
          float2 w = cscale(v[j], zf);
          if (mi) w = cmuli(w);
          if (ok) d[(size_t)fft_out_index<N, V>(p, j) * nhp] = w;
        }
      }
      __syncthreads();
    }
  }
  if (kStore && tid == 0) bulk_wait_all();
}

// One x/y tile width: staged tile + exchange + twiddles + multipliers +
// alignment slack, and the block size.
template <int N, int TC, int V = 0> struct CfgXY {
  static constexpr int E = Shape<N, V>::E, P = Shape<N, V>::P, P1 = Shape<N, V>::P1, NTW = Shape<N, V>::kTw;
  static constexpr size_t smem = (size_t)N * TC * 8 + (size_t)XLayoutCols<E, P, TC, P1>::kSize * 8 +
                                 (size_t)NTW * 8 + (size_t)3 * N * 4 + 128;
  static constexpr int threads = TC * P;
};

// The x/y tile widths a plan may run (the autotuner's candidates): the
// default and half of it while a TMA box row stays at least 64 bytes.  Every
// width computes each column's transform with the same arithmetic, so the
// choice changes timings only.
#ifndef PIN_TC_LONG
#define PIN_TC_LONG 16
#endif
// default columns per x/y tile for P threads per line (a TMA box row is TC x 8 bytes)
constexpr int default_tc(int P) { return P >= 16 ? PIN_TC_LONG : (P >= 8 ? 16 : (P == 4 ? 32 : 64)); }
template <int N, int V = 0> struct Tiles {
  static constexpr int T0 = default_tc(Shape<N, V>::P);
  static constexpr int T1 = T0 / 2 >= 8 ? T0 / 2 : T0;
};

template <int N, int TC, int V>
static cudaError_t set_attrs_xy() {
  constexpr int smem = (int)CfgXY<N, TC, V>::smem;
  cudaError_t e = cudaFuncSetAttribute(k_pass_x<N, TC, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_pass_y<N, TC, false, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_pass_y<N, TC, true, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

// both tile widths of one radix schedule
template <int N, int V>
static cudaError_t set_attrs_xy_all() {
  cudaError_t e = set_attrs_xy<N, Tiles<N, V>::T0, V>();
  if (e != cudaSuccess) return e;
  if constexpr (Tiles<N, V>::T1 != Tiles<N, V>::T0) e = set_attrs_xy<N, Tiles<N, V>::T1, V>();
  return e;
}

// Persistent grid: as many blocks as fit on the device at once, at most one
// per tile.
template <class K>
static unsigned persistent_grid(K kernel, int threads, size_t smem, long ntiles) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
  long g = (long)std::max(1, sms) * std::max(1, per_sm);
  return (unsigned)std::min<long>(g, std::max<long>(1, ntiles));
}

template <int N, int TC, int V>
static cudaError_t run_x(const ArgsX& a_in, cudaStream_t st) {
  using C = CfgXY<N, TC, V>;
  ArgsX a = a_in;
  if (PIN_X_TMASTORE) {
    // output maps: the same geometry as the source map, one per output
    for (int f = 0; f < a.nout; ++f) {
      const cudaError_t e = make_tmap_x(&a.tm_out[f], a.dst[f], N, a.ny, a.nhp, a.batch, TC);
      if (e != cudaSuccess) return e;
    }
  }
  const long ntiles = (((long)a.ny * a.nhp + TC - 1) / TC) * a.batch;
  const unsigned grid = persistent_grid(k_pass_x<N, TC, V>, C::threads, C::smem, ntiles);
  k_pass_x<N, TC, V><<<grid, C::threads, C::smem, st>>>(a);
  return cudaGetLastError();
}

template <int N, int TC, int V>
static cudaError_t run_y(const ArgsY& a, cudaStream_t st) {
  using C = CfgXY<N, TC, V>;
  const long ntiles = (long)a.nx * a.batch * ((a.nhp + TC - 1) / TC);
  bool dual = false;
  for (int o = 0; o < a.nout; ++o) dual = dual || a.dst2[o] != nullptr;
  if (PIN_Y_TMASTORE && !dual) {
    // output maps: rows (x, ky) of nhp values, boxes of the staged tile's rows
    ArgsY b = a;
    for (int o = 0; o < b.nout; ++o) {
      const cudaError_t e = make_tmap_rows(&b.tm_out[o], b.dst[o], b.nhp, (long long)b.nx * b.batch * N, TC,
                                           Stage<N>::kRows);
      if (e != cudaSuccess) return e;
    }
    const unsigned grid = persistent_grid(k_pass_y<N, TC, false, V>, C::threads, C::smem, ntiles);
    k_pass_y<N, TC, false, V><<<grid, C::threads, C::smem, st>>>(b);
    return cudaGetLastError();
  }
  if (dual) {
    const unsigned grid = persistent_grid(k_pass_y<N, TC, true, V>, C::threads, C::smem, ntiles);
    k_pass_y<N, TC, true, V><<<grid, C::threads, C::smem, st>>>(a);
  } else {
    const unsigned grid = persistent_grid(k_pass_y<N, TC, false, V>, C::threads, C::smem, ntiles);
    k_pass_y<N, TC, false, V><<<grid, C::threads, C::smem, st>>>(a);
  }
  return cudaGetLastError();
}

// launch with a tile width that is one of Tiles<N, V> (anything else: the default)
template <int N, int V>
static cudaError_t launch_x_v(int tc, const ArgsX& a, cudaStream_t st) {
  return tc == Tiles<N, V>::T1 ? run_x<N, Tiles<N, V>::T1, V>(a, st) : run_x<N, Tiles<N, V>::T0, V>(a, st);
}
template <int N, int V>
static cudaError_t launch_y_v(int tc, const ArgsY& a, cudaStream_t st) {
  return tc == Tiles<N, V>::T1 ? run_y<N, Tiles<N, V>::T1, V>(a, st) : run_y<N, Tiles<N, V>::T0, V>(a, st);
}

template <int N, int V>
static PassShape xy_shape_of() {
  using S = Shape<N, V>;
  constexpr int TC = Tiles<N, V>::T0;
  return PassShape{S::E, S::P, S::P1, S::P2, TC, 0, CfgXY<N, TC, V>::smem, 0, CfgXY<N, TC, V>::threads, 0};
}


}  // namespace pin
