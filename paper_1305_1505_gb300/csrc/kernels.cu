// The three passes of one smoothing radius (Sec. 2.1.1, Collapse times):
//   x pass  : filter (x factors of W and k_i k_j) fused into the inverse DFT
//             along x, three outputs;
//   y pass  : y factors and the inverse DFT along y, six outputs;
//   z pass  : z factors, complex-to-real inverse DFT along z of the six
//             Hessian components (two per complex transform), then per grid
//             point the eigenvalues, the collapse time F = 1/D_c and the
//             running maximum F_max with its radius index, written in place.
// Each thread block owns a tile of lines; every line is transformed by the
// register FFT of fft.cuh (two levels with one shared-memory exchange, or,
// for 384 and 768 points, three levels with two).  The x and y passes run one
// of two compiled tile widths, chosen per plan (pin_autotune).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <mutex>

#include "collapse.cuh"
#include "collapse_x2.cuh"
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
#ifndef PIN_Z_MINB
#define PIN_Z_MINB 2
#endif
// Independent particles per iteration of the collapse loop.
#ifndef PIN_Z_ILP
#define PIN_Z_ILP 2
#endif
#ifndef PIN_Z_MINB3
#define PIN_Z_MINB3 4
#endif
// Three-level lines hold half the registers per thread: the z pass is sized
// for more resident blocks.
template <int N, int TC = 16> struct MinBlocks {
  // three-level x/y blocks (TC columns x P threads) are sized for 512
  // resident threads per SM
  static constexpr int xy = Shape<N>::P2 > 1 ? 512 / (TC * Shape<N>::P) : (N >= 384 ? PIN_XY_MINB : 1);
  static constexpr int z = Shape<N>::P2 > 1 ? PIN_Z_MINB3 : (N >= 384 ? PIN_Z_MINB : 1);
};

// ---------------------------------------------------------------- x pass --
// Lines along x: column index col in [0, N*nhp) enumerates (ky, kz); element
// (kx, col) sits at kx*N*nhp + col, so a row of TC columns is contiguous.  A
// persistent block walks column tiles; the staged Phi0 tile serves all
// outputs, and the next tile is requested as soon as the last output has read
// the current one into registers.
template <int N, int TC>
__global__ void __launch_bounds__(TC* Shape<N>::P, MinBlocks<N, TC>::xy) k_pass_x(const __grid_constant__ ArgsX a) {
  constexpr int E = Shape<N>::E, P = Shape<N>::P, NTW = Shape<N>::kTw;
  using L = XLayoutCols<E, P, TC, Shape<N>::P1>;
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
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    if (!stage_ready(bar, parity, a.err, a.wait_cycles)) return;
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
      fft_line<N, L>(v, p, c, s_x, s_tw);
      float2* d = s_dst[f] + rbase + (ok ? col : 0);
#pragma unroll
      for (int j = 0; j < E; ++j)
        if (ok) d[(size_t)fft_out_index<N>(p, j) * ncols] = v[j];
      __syncthreads();
    }
  }
}

// ---------------------------------------------------------------- y pass --
// Lines along y: a tile is TC consecutive kz of one x plane; element
// (ky, kz) of plane x sits at (x*N + ky)*nhp + kz.  Columns past nhp are
// zero-filled by the tensor map and not stored.
template <int N, int TC, bool DUAL>
__global__ void __launch_bounds__(TC* Shape<N>::P, MinBlocks<N, TC>::xy) k_pass_y(const __grid_constant__ ArgsY a) {
  constexpr int E = Shape<N>::E, P = Shape<N>::P, NTW = Shape<N>::kTw;
  using L = XLayoutCols<E, P, TC, Shape<N>::P1>;
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
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int x = tile / ktiles, kz = (tile % ktiles) * TC + c;
    const bool ok = kz < nhp;
    const size_t base = (size_t)x * N * nhp + (ok ? kz : 0);
#pragma unroll 1
    for (int o = 0; o < nout; ++o) {
      if (o == 0 || s_sel[o] != s_sel[o - 1]) {
        if (!stage_ready(bar, parity, a.err, a.wait_cycles)) return;
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
      fft_line<N, L>(v, p, c, s_x, s_tw);
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
          const size_t off = (size_t)fft_out_index<N>(p, j) * nhp;
          float2 w = cscale(v[j], zf);
          if (mi) w = cmuli(w);
          if (ok) d[off] = w;
          if (two) {
            float2 w2 = cscale(v[j], zf2);
            if (mi2) w2 = cmuli(w2);
            d2[off] = w2;
          }
        }
      } else {
#pragma unroll
        for (int j = 0; j < E; ++j) {
          float2 w = cscale(v[j], zf);
          if (mi) w = cmuli(w);
          if (ok) d[(size_t)fft_out_index<N>(p, j) * nhp] = w;
        }
      }
      __syncthreads();
    }
  }
}

// Stride (floats) of one real field line in the z pass's shared buffer, padded
// so that the stores of the transform outputs spread over the banks: two-level
// lines write runs of P consecutive z per pair-column (offset P/2), three-level
// lines write z = k1 + E (k2a + P2 k2b) (offset 2, so that the two
// pair-columns of a 16-thread-line warp land on disjoint banks).
template <int N> __host__ __device__ constexpr int field_stride() {
  return Shape<N>::P2 > 1 ? N + 2 : N + (Shape<N>::P >= 2 ? Shape<N>::P / 2 : 1);
}

// ---------------------------------------------------------------- z pass --
// Lines along z: line index l = x*N + y, the half line src[f][l*nhp + kz],
// kz in [0, N/2], is contiguous.  Fields are paired (A + iB) into one complex
// length-N transform whose real and imaginary parts are the two real lines.
// NP pairs per line: 3 (the six Hessian components) or 5 (plus the three
// smoothed displacement components, kept for the velocity at R_max).
// FUSE: the collapse time and the running maximum of every particle follow
// its eigenvalues in this kernel (no eigenvalue round trip through memory);
// otherwise the eigenvalues go to lam_out for k_roots.  SRC: instead, the
// second-order LPT source S = sum_{i<j} (phi_ii phi_jj - phi_ij^2) of every
// particle goes to out[0] (a real field).
template <int N, int LINES, bool DUMP, int NP, bool FUSE, bool SRC = false>
__global__ void __launch_bounds__(NP * LINES * Shape<N>::P, MinBlocks<N>::z) k_pass_z(ArgsZ a) {
  constexpr int E = Shape<N>::E, P = Shape<N>::P, NTW = Shape<N>::kTw;
  constexpr int NC = NP * LINES;  // pair-columns of the block
  constexpr int NF = 2 * NP;      // field slots per line
  using L = XLayoutLines<E, P, NC, Shape<N>::P1>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float2* s_x = reinterpret_cast<float2*>(smem_raw);
  constexpr int kFS = field_stride<N>();
  constexpr int kXBytes = L::kSize * 8, kFBytes = LINES * NF * kFS * 4;
  constexpr int kBufBytes = kXBytes > kFBytes ? kXBytes : kFBytes;
  float2* s_tw = reinterpret_cast<float2*>(reinterpret_cast<char*>(smem_raw) + kBufBytes);
  float* s_f = reinterpret_cast<float*>(smem_raw);
  const int nthreads = NC * P;
  const int tid = threadIdx.x;
  for (int i = tid; i < NTW; i += nthreads) s_tw[i] = a.tw[i];
  __syncthreads();

  const int npairs = (a.nfields + 1) / 2;
  const int c = tid / P, p = tid % P;
  const int ln = c / NP, pair = c % NP;
  const int nlines = a.nlines;
  const int line = blockIdx.x * LINES + ln;
  const bool active = pair < npairs && line < nlines;
  const int fa = 2 * pair, fb = 2 * pair + 1;
  const bool hasb = active && fb < a.nfields;
  const int nhp = a.nhp;

  float2 v[E];
  {
    const float2* A = active ? a.src[fa] + (size_t)line * nhp : nullptr;
    const float2* B = hasb ? a.src[fb] + (size_t)line * nhp : nullptr;
#pragma unroll
    for (int t = 0; t < E; ++t) {
      const int n = p + P * t;
      // slot t holds n in [P t, P t + P): wholly below N/2, wholly above, or
      // straddling it; the first two are decided at compile time
      const bool below = P * t + P - 1 < N / 2, above = P * t > N / 2;
      const int m = below ? n : (above ? N - n : (n <= N / 2 ? n : N - n));
      const bool conj = !below && (above || n > N / 2);
      const bool real = below ? (t == 0 && p == 0) : (!above && (n == N / 2 || n == 0));
      float2 xa = make_float2(0.f, 0.f), xb = make_float2(0.f, 0.f);
      if (active) xa = __ldg(A + m);
      if (hasb) xb = __ldg(B + m);
      if (real) {
        xa.y = 0.f;
        xb.y = 0.f;
      } else if (conj) {
        xa = cconj(xa);
        xb = cconj(xb);
      }
      v[t] = make_float2(xa.x - xb.y, xa.y + xb.x);  // A + iB
    }
  }
  fft_line<N, L, 32 % Shape<N>::P == 0>(v, p, c, s_x, s_tw);

  if constexpr (DUMP) {
    if (active) {
      float* oa = a.out[fa] + (size_t)line * N;
      float* ob = hasb ? a.out[fb] + (size_t)line * N : nullptr;
#pragma unroll
      for (int j = 0; j < E; ++j) {
        const int z = fft_out_index<N>(p, j);
        oa[z] = v[j].x;
        if (hasb) ob[z] = v[j].y;
      }
    }
    return;
  } else {
    __syncthreads();  // exchange buffer becomes the field buffer
    if (pair < npairs) {
#pragma unroll
      for (int j = 0; j < E; ++j) {
        const int z = fft_out_index<N>(p, j);
        s_f[(ln * NF + fa) * kFS + z] = v[j].x;
        s_f[(ln * NF + fb) * kFS + z] = v[j].y;
      }
    }
    __syncthreads();
    constexpr int kPts = LINES * N;
    const size_t total = (size_t)nlines * N;
    if constexpr (SRC) {
      for (int pt = tid; pt < kPts; pt += nthreads) {
        const int l = pt / N, z = pt % N;
        const int gl = blockIdx.x * LINES + l;
        if (gl >= nlines) continue;
        float h[6];
#pragma unroll
        for (int f = 0; f < 6; ++f) h[f] = s_f[(l * NF + f) * kFS + z];
        a.out[0][(size_t)gl * N + z] =
            h[0] * h[1] + h[0] * h[2] + h[1] * h[2] - h[3] * h[3] - h[4] * h[4] - h[5] * h[5];
      }
    } else if constexpr (FUSE && PIN_Z_ILP % 2 == 0) {
      // eigenvalues, collapse time and running maximum of PIN_Z_ILP particles
      // per thread and iteration, held two by two in the lanes of packed
      // pairs (NPR independent pairs, so that their dependency chains
      // interleave)
      constexpr int NPR = PIN_Z_ILP / 2;
      const CollapseConsts<float> ccf{a.dcorr_f, a.correction};
      for (int pt0 = tid; pt0 < kPts; pt0 += 2 * NPR * nthreads) {
        int q[NPR][2], lz[NPR][2];
        bool valid[NPR][2];
        float fm[NPR][2];
        float2 lam[NPR][3];
#pragma unroll
        for (int r = 0; r < NPR; ++r) {
          float2 h[6];
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const int pt = pt0 + (2 * r + u) * nthreads;
            const int l = pt / N, z = pt % N;
            const int gl = blockIdx.x * LINES + l;
            valid[r][u] = pt < kPts && gl < nlines;
            q[r][u] = gl * N + z;  // < 2^31: checked at plan creation
            lz[r][u] = (l * NF) * kFS + z;
#pragma unroll
            for (int f = 0; f < 6; ++f) {
              const float v = valid[r][u] ? s_f[lz[r][u] + f * kFS] : 0.f;
              if (u) h[f].y = v;
              else h[f].x = v;
            }
          }
          const float2 rabs = eig3_x2(h, lam[r]);
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            fm[r][u] = valid[r][u] ? a.fmax[q[r][u]] : 0.f;
            if (valid[r][u] && (u ? rabs.y : rabs.x) > 1.f - a.tau_eig) {
              atomicAdd(a.counters + 0, 1ull);
              const unsigned slot = atomicAdd(a.redo_count, 1u);
              if (slot < a.redo_cap) {
                RedoEntry e;
                e.q = q[r][u];
#pragma unroll
                for (int f = 0; f < 6; ++f) e.h[f] = u ? h[f].y : h[f].x;
                e.kind = 0;
                a.redo_list[slot] = e;
                if constexpr (NP == 5) {
#pragma unroll
                  for (int cpt = 0; cpt < 3; ++cpt)
                    a.psi_out[cpt * total + q[r][u]] = s_f[lz[r][u] + (6 + cpt) * kFS];
                }
                valid[r][u] = false;  // the redo kernel updates this particle
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                  if (u) lam[r][k].y = 0.f;
                  else lam[r][k].x = 0.f;
                }
              } else {
                atomicAdd(a.counters + 2, 1ull);  // queue full: keep the FP32 eigenvalues
              }
            }
          }
        }
        // lanes that cannot beat their running maximum (the radii run
        // smallest first, so most particles reach F_max early) or that the
        // FP64 redo finishes skip the root solve; a pair solves only if one of
        // its lanes needs it
        CollapseStateX2 csx[NPR];
        unsigned done[NPR];
#pragma unroll
        for (int r = 0; r < NPR; ++r) {
          float2 c0[3];
          collapse_prep_x2(lam[r], ccf, csx[r], c0);
          done[r] = cannot_beat_x2(c0, csx[r], make_float2(fm[r][0], fm[r][1])) | (valid[r][0] ? 0u : 1u) |
                    (valid[r][1] ? 0u : 2u);
          if (done[r] != 3u) collapse_root_x2(c0, csx[r]);
        }
#pragma unroll
        for (int r = 0; r < NPR; ++r)
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            if ((done[r] >> u) & 1u) continue;
            CollapseState<float> cs = lane_state(csx[r], u);
            if (cs.need[0] || cs.need[1]) collapse_rare<float>(cs);
            const int qq = q[r][u];
            const float F = cs.best + cs.corr;
            if (cs.kappa < a.tau_root) {
              atomicAdd(a.counters + 1, 1ull);
              const unsigned slot = atomicAdd(a.redo_count, 1u);
              if (slot < a.redo_cap) {
                RedoEntry e;
                e.q = qq;
#pragma unroll
                for (int k = 0; k < 3; ++k) e.h[k] = u ? lam[r][k].y : lam[r][k].x;
                e.h[3] = e.h[4] = e.h[5] = 0.f;
                e.kind = 1;
                a.redo_list[slot] = e;
                if constexpr (NP == 5) {
#pragma unroll
                  for (int cpt = 0; cpt < 3; ++cpt) a.psi_out[cpt * total + qq] = s_f[lz[r][u] + (6 + cpt) * kFS];
                }
                continue;
              }
              atomicAdd(a.counters + 2, 1ull);  // queue full: keep the FP32 value
            }
            if (F > fm[r][u] || (F == fm[r][u] && F > 0.f && a.scale < a.idx[qq])) {
              a.fmax[qq] = F;
              a.idx[qq] = a.scale;
              if constexpr (NP == 5) {
#pragma unroll
                for (int cpt = 0; cpt < 3; ++cpt) a.vstate[cpt * total + qq] = s_f[lz[r][u] + (6 + cpt) * kFS];
              }
            }
          }
      }
    } else if constexpr (FUSE) {
      // eigenvalues, collapse time and running maximum, PIN_Z_ILP particles
      // per thread and iteration
      constexpr int U = PIN_Z_ILP;
      const CollapseConsts<float> ccf{a.dcorr_f, a.correction};
      for (int pt0 = tid; pt0 < kPts; pt0 += U * nthreads) {
        float lam[U][3], fm[U];
        bool valid[U];
        int q[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int pt = pt0 + u * nthreads;
          const int l = pt / N, z = pt % N;
          const int gl = blockIdx.x * LINES + l;
          valid[u] = pt < kPts && gl < nlines;
          q[u] = gl * N + z;  // < 2^31: checked at plan creation
          fm[u] = 0.f;
          lam[u][0] = lam[u][1] = lam[u][2] = 0.f;
          if (valid[u]) {
            float h[6];
#pragma unroll
            for (int f = 0; f < 6; ++f) h[f] = s_f[(l * NF + f) * kFS + z];
            const float rabs = eig3<float>(h, lam[u]);
            fm[u] = a.fmax[q[u]];
            if (rabs > 1.f - a.tau_eig) {
              atomicAdd(a.counters + 0, 1ull);
              const unsigned slot = atomicAdd(a.redo_count, 1u);
              if (slot < a.redo_cap) {
                RedoEntry e;
                e.q = q[u];
#pragma unroll
                for (int f = 0; f < 6; ++f) e.h[f] = h[f];
                e.kind = 0;
                a.redo_list[slot] = e;
                if constexpr (NP == 5) {
#pragma unroll
                  for (int cpt = 0; cpt < 3; ++cpt)
                    a.psi_out[cpt * total + q[u]] = s_f[(l * NF + 6 + cpt) * kFS + z];
                }
                valid[u] = false;  // the redo kernel updates this particle
                lam[u][0] = lam[u][1] = lam[u][2] = 0.f;
              } else {
                atomicAdd(a.counters + 2, 1ull);  // queue full: keep the FP32 eigenvalues
              }
            }
          }
        }
        CollapseState<float> cs[U];
#pragma unroll
        for (int u = 0; u < U; ++u) collapse_main<float>(lam[u], ccf, cs[u]);
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (cs[u].need[0] || cs[u].need[1]) collapse_rare<float>(cs[u]);
#pragma unroll
        for (int u = 0; u < U; ++u) {
          if (!valid[u]) continue;
          const int pt = pt0 + u * nthreads;
          const int l = pt / N, z = pt % N;
          const float F = cs[u].best + cs[u].corr;
          if (cs[u].kappa < a.tau_root) {
            atomicAdd(a.counters + 1, 1ull);
            const unsigned slot = atomicAdd(a.redo_count, 1u);
            if (slot < a.redo_cap) {
              RedoEntry e;
              e.q = q[u];
              e.h[0] = lam[u][0];
              e.h[1] = lam[u][1];
              e.h[2] = lam[u][2];
              e.h[3] = e.h[4] = e.h[5] = 0.f;
              e.kind = 1;
              a.redo_list[slot] = e;
              if constexpr (NP == 5) {
#pragma unroll
                for (int cpt = 0; cpt < 3; ++cpt)
                  a.psi_out[cpt * total + q[u]] = s_f[(l * NF + 6 + cpt) * kFS + z];
              }
              continue;
            }
            atomicAdd(a.counters + 2, 1ull);  // queue full: keep the FP32 value
          }
          if (F > fm[u] || (F == fm[u] && F > 0.f && a.scale < a.idx[q[u]])) {
            a.fmax[q[u]] = F;
            a.idx[q[u]] = a.scale;
            if constexpr (NP == 5) {
#pragma unroll
              for (int cpt = 0; cpt < 3; ++cpt) a.vstate[cpt * total + q[u]] = s_f[(l * NF + 6 + cpt) * kFS + z];
            }
          }
        }
      }
    } else {
      // eigenvalues of every particle of the block's lines; the collapse time
      // and the running maximum follow in k_roots
      for (int pt = tid; pt < kPts; pt += nthreads) {
        const int l = pt / N, z = pt % N;
        const int gl = blockIdx.x * LINES + l;
        if (gl >= nlines) continue;
        float h[6], lam[3];
#pragma unroll
        for (int f = 0; f < 6; ++f) h[f] = s_f[(l * NF + f) * kFS + z];
        const float rabs = eig3<float>(h, lam);
        const int q = gl * N + z;  // < 2^31: checked at plan creation
        if (rabs > 1.f - a.tau_eig) {
          atomicAdd(a.counters + 0, 1ull);
          const unsigned slot = atomicAdd(a.redo_count, 1u);
          if (slot < a.redo_cap) {
            RedoEntry e;
            e.q = q;
#pragma unroll
            for (int f = 0; f < 6; ++f) e.h[f] = h[f];
            e.kind = 0;
            a.redo_list[slot] = e;
            lam[0] = lam[1] = lam[2] = __int_as_float(0x7fc00000);  // NaN: skipped by k_roots
          } else {
            atomicAdd(a.counters + 2, 1ull);  // queue full: keep the FP32 eigenvalues
          }
        }
        a.lam_out[q] = lam[0];
        a.lam_out[total + q] = lam[1];
        a.lam_out[2 * total + q] = lam[2];
        if constexpr (NP == 5) {
          // smoothed displacement of this radius, copied to the state by k_roots
          // when F_max moves here
#pragma unroll
          for (int cpt = 0; cpt < 3; ++cpt) a.psi_out[cpt * total + q] = s_f[(l * NF + 6 + cpt) * kFS + z];
        }
      }
    }
  }
}

// --------------------------------------------------- forward z (real in) --
// T(x, y, kz) = sum_z s(x, y, z) exp(+2 pi i z kz / N) for kz in [0, N/2] of
// every real line s (the inverse-sign transform of real data; its conjugate is
// the forward transform).  Two lines A, B ride one complex transform of A + iB,
// Z = T_A + i T_B, and are separated with T_A(k) = (Z(k) + conj Z(N-k)) / 2,
// T_B(k) = (Z(k) - conj Z(N-k)) / 2i.  Output in the padded half-spectrum
// layout (kz stride nhp, pad modes zero).
template <int N, int NC>
__global__ void __launch_bounds__(NC * Shape<N>::P) k_fwd_z(const float* __restrict__ src, float2* dst, int nlines,
                                                          int nhp, const float2* tw) {
  constexpr int E = Shape<N>::E, P = Shape<N>::P, NTW = Shape<N>::kTw;
  using L = XLayoutLines<E, P, NC, Shape<N>::P1>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float2* s_x = reinterpret_cast<float2*>(smem_raw);
  constexpr int kXBytes = L::kSize * 8, kZBytes = NC * N * 8;
  constexpr int kBufBytes = kXBytes > kZBytes ? kXBytes : kZBytes;
  float2* s_tw = reinterpret_cast<float2*>(smem_raw + kBufBytes);
  float2* s_z = s_x;  // after the transform: Z of each pair, [NC][N]
  const int tid = threadIdx.x, c = tid / P, p = tid % P;
  for (int i = tid; i < NTW; i += NC * P) s_tw[i] = tw[i];
  __syncthreads();
  const int la = 2 * (blockIdx.x * NC + c);  // lines la, la + 1
  const bool active = la < nlines;
  float2 v[E];
  const float* A = src + (size_t)(active ? la : 0) * N;
#pragma unroll
  for (int t = 0; t < E; ++t) {
    const int n = p + P * t;
    v[t] = active ? make_float2(__ldg(A + n), __ldg(A + N + n)) : make_float2(0.f, 0.f);
  }
  fft_line<N, L, 32 % Shape<N>::P == 0>(v, p, c, s_x, s_tw);
  __syncthreads();
#pragma unroll
  for (int j = 0; j < E; ++j) s_z[c * N + fft_out_index<N>(p, j)] = v[j];
  __syncthreads();
  if (!active) return;
  float2* oa = dst + (size_t)la * nhp;
  float2* ob = oa + nhp;
  for (int k = p; k < nhp; k += P) {
    float2 ta = make_float2(0.f, 0.f), tb = make_float2(0.f, 0.f);
    if (k <= N / 2) {
      const float2 zk = s_z[c * N + k], zm = s_z[c * N + (k == 0 ? 0 : N - k)];
      ta = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
      tb = make_float2(0.5f * (zk.y + zm.y), 0.5f * (zm.x - zk.x));
    }
    oa[k] = ta;
    ob[k] = tb;
  }
}

// Phi2(k) = scale conj(T(k)) / k^2 on the padded half-spectrum (k = 0 and
// pad modes zero): with T the inverse-sign transform of the 2LPT source, the
// potential whose gradient i k Phi2 is the second-order displacement.
// Cubic cells: the box side along x is `box`, L_y = box ny / nx, L_z = box nz / nx.
__global__ void k_phi2(const float2* __restrict__ T, float2* out, int nx, int ny, int nz, int nhp, double box,
                       float scale) {
  const size_t total = (size_t)nx * ny * nhp;
  const float kfx = (float)(2.0 * M_PI / box), kfy = (float)(2.0 * M_PI / (ny == nx ? box : box * ny / nx)),
              kfz = (float)(2.0 * M_PI / (nz == nx ? box : box * nz / nx));
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int iz = (int)(i % nhp);
    const size_t row = i / nhp;
    const int iy = (int)(row % ny), ix = (int)(row / ny);
    float2 r = make_float2(0.f, 0.f);
    if (iz <= nz / 2) {
      const int sx = ix < nx / 2 ? ix : ix - nx, sy = iy < ny / 2 ? iy : iy - ny;
      const float kx = kfx * sx, ky = kfy * sy, kz = kfz * iz;
      const float k2 = kx * kx + ky * ky + kz * kz;
      if (k2 > 0.f) {
        const float2 t = T[i];
        const float f = scale / k2;
        r = make_float2(f * t.x, -f * t.y);
      }
    }
    out[i] = r;
  }
}

// ------------------------------------------------------------- root pass --
// Per particle: the collapse time F from its eigenvalues (collapse.cuh), and
// the running maximum F_max with its radius index, updated in place.  Few
// registers, so many warps hide the latency of the dependent root iteration;
// PIN_Z_ILP particles per thread and iteration.
template <bool VEL>
__global__ void __launch_bounds__(256) k_roots(ArgsZ a) {
  constexpr int U = PIN_Z_ILP;
  const int total = a.npart;
  const float* L0 = a.lam_out;
  const float* L1 = a.lam_out + total;
  const float* L2 = a.lam_out + 2 * (size_t)total;
  CollapseConsts<float> ccf{a.dcorr_f, a.correction};
  const int stride = gridDim.x * blockDim.x;
  if constexpr (U == 2) {
    // two particles per thread in the lanes of packed pairs
    for (int q0 = blockIdx.x * blockDim.x + threadIdx.x; q0 < total; q0 += 2 * stride) {
      float2 lam[3];
      float fm[2];
      bool valid[2];
      int q[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        q[u] = q0 + u * stride;
        const bool in = q[u] < total;
        float l0 = in ? __ldg(L0 + q[u]) : 0.f, l1 = in ? __ldg(L1 + q[u]) : 0.f, l2 = in ? __ldg(L2 + q[u]) : 0.f;
        fm[u] = in ? a.fmax[q[u]] : 0.f;
        valid[u] = in && !isnan(l0);  // NaN: queued by the z pass
        if (!valid[u]) l0 = l1 = l2 = 0.f;
        if (u) {
          lam[0].y = l0; lam[1].y = l1; lam[2].y = l2;
        } else {
          lam[0].x = l0; lam[1].x = l1; lam[2].x = l2;
        }
      }
      CollapseStateX2 csx;
      float2 c0[3];
      collapse_prep_x2(lam, ccf, csx, c0);
      const unsigned done = cannot_beat_x2(c0, csx, make_float2(fm[0], fm[1])) | (valid[0] ? 0u : 1u) |
                            (valid[1] ? 0u : 2u);
      if (done != 3u) collapse_root_x2(c0, csx);
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        if ((done >> u) & 1u) continue;
        CollapseState<float> cs = lane_state(csx, u);
        if (cs.need[0] || cs.need[1]) collapse_rare<float>(cs);
        const float F = cs.best + cs.corr;
        if (cs.kappa < a.tau_root) {
          atomicAdd(a.counters + 1, 1ull);
          const unsigned slot = atomicAdd(a.redo_count, 1u);
          if (slot < a.redo_cap) {
            RedoEntry e;
            e.q = q[u];
#pragma unroll
            for (int k = 0; k < 3; ++k) e.h[k] = u ? lam[k].y : lam[k].x;
            e.h[3] = e.h[4] = e.h[5] = 0.f;
            e.kind = 1;
            a.redo_list[slot] = e;
            continue;  // the redo kernel updates this particle
          }
          atomicAdd(a.counters + 2, 1ull);  // queue full: keep the FP32 value
        }
        if (F > fm[u] || (F == fm[u] && F > 0.f && a.scale < a.idx[q[u]])) {
          a.fmax[q[u]] = F;
          a.idx[q[u]] = a.scale;
          if constexpr (VEL) {
#pragma unroll
            for (int cpt = 0; cpt < 3; ++cpt)
              a.vstate[(size_t)cpt * total + q[u]] = a.psi_out[(size_t)cpt * total + q[u]];
          }
        }
      }
    }
  } else {
  for (int q0 = blockIdx.x * blockDim.x + threadIdx.x; q0 < total; q0 += U * stride) {
    float lam[U][3], fm[U];
    bool valid[U];
    int q[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      q[u] = q0 + u * stride;
      const bool in = q[u] < total;
      lam[u][0] = in ? __ldg(L0 + q[u]) : 0.f;
      lam[u][1] = in ? __ldg(L1 + q[u]) : 0.f;
      lam[u][2] = in ? __ldg(L2 + q[u]) : 0.f;
      fm[u] = in ? a.fmax[q[u]] : 0.f;
      valid[u] = in && !isnan(lam[u][0]);  // NaN: queued by the z pass
      if (!valid[u]) lam[u][0] = lam[u][1] = lam[u][2] = 0.f;
    }
    CollapseState<float> cs[U];
#pragma unroll
    for (int u = 0; u < U; ++u) collapse_main<float>(lam[u], ccf, cs[u]);
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (cs[u].need[0] || cs[u].need[1]) collapse_rare<float>(cs[u]);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (!valid[u]) continue;
      const float F = cs[u].best + cs[u].corr;
      if (cs[u].kappa < a.tau_root) {
        atomicAdd(a.counters + 1, 1ull);
        const unsigned slot = atomicAdd(a.redo_count, 1u);
        if (slot < a.redo_cap) {
          RedoEntry e;
          e.q = q[u];
          e.h[0] = lam[u][0];
          e.h[1] = lam[u][1];
          e.h[2] = lam[u][2];
          e.h[3] = e.h[4] = e.h[5] = 0.f;
          e.kind = 1;
          a.redo_list[slot] = e;
          continue;  // the redo kernel updates this particle
        }
        atomicAdd(a.counters + 2, 1ull);  // queue full: keep the FP32 value
      }
      if (F > fm[u] || (F == fm[u] && F > 0.f && a.scale < a.idx[q[u]])) {
        a.fmax[q[u]] = F;
        a.idx[q[u]] = a.scale;
        if constexpr (VEL) {
#pragma unroll
          for (int cpt = 0; cpt < 3; ++cpt)
            a.vstate[(size_t)cpt * total + q[u]] = a.psi_out[(size_t)cpt * total + q[u]];
        }
      }
    }
  }
  }
}

cudaError_t launch_roots(const ArgsZ& a, cudaStream_t st) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long need = ((long)a.npart + 255) / 256;
  const unsigned grid = (unsigned)std::max<long>(1, std::min<long>(need, (long)sms * 8));
  if (a.vstate) k_roots<true><<<grid, 256, 0, st>>>(a);
  else k_roots<false><<<grid, 256, 0, st>>>(a);
  return cudaGetLastError();
}

// FP64 redo of the queued particles of one radius (grid-stride; each particle
// appears once per radius, so the in-place update has no race).
__global__ void __launch_bounds__(128) k_redo64(ArgsZ a) {
  const unsigned cnt = *a.redo_count;
  const unsigned n = cnt < a.redo_cap ? cnt : a.redo_cap;
  CollapseConsts<double> ccd{a.dcorr_d, a.correction};
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const RedoEntry e = a.redo_list[i];
    double h[6], lam[3], kap;
#pragma unroll
    for (int f = 0; f < 6; ++f) h[f] = (double)e.h[f];
    if (e.kind == 0) {
      eig3<double>(h, lam);
    } else {
      lam[0] = h[0];
      lam[1] = h[1];
      lam[2] = h[2];
    }
    const float F = (float)collapse_from_eigs<double>(lam, ccd, kap);
    const float fm = a.fmax[e.q];
    if (F > fm || (F == fm && F > 0.f && a.scale < a.idx[e.q])) {
      a.fmax[e.q] = F;
      a.idx[e.q] = a.scale;
      if (a.vstate) {
        const size_t total = (size_t)a.npart;
#pragma unroll
        for (int cpt = 0; cpt < 3; ++cpt) a.vstate[cpt * total + e.q] = a.psi_out[cpt * total + e.q];
      }
    }
  }
}

cudaError_t launch_redo(const ArgsZ& a, cudaStream_t st) {
  k_redo64<<<2 * 152, 128, 0, st>>>(a);
  return cudaGetLastError();
}

// -------------------------------------------------------------- dispatch --

template <int N> struct Cfg {
  static constexpr int E = Shape<N>::E, P = Shape<N>::P, P1 = Shape<N>::P1, NTW = Shape<N>::kTw;
  // columns per x/y tile (a TMA box row is TC x 8 bytes)
#ifndef PIN_TC_LONG
#define PIN_TC_LONG 16
#endif
  static constexpr int TC = P >= 16 ? PIN_TC_LONG : (P >= 8 ? 16 : (P == 4 ? 32 : 64));
  static constexpr int LINES = P >= 64 ? 1 : 64 / P;
  // the root solve runs inside the z pass where its transform leaves the
  // registers for it (three-level lines)
#ifndef PIN_Z_FUSE
  static constexpr bool FUSE = Shape<N>::P2 > 1;
#else
  static constexpr bool FUSE = PIN_Z_FUSE != 0;
#endif
  static constexpr size_t xz = (size_t)XLayoutLines<E, P, 3 * LINES, P1>::kSize * 8;
  static constexpr size_t fz = (size_t)LINES * 6 * field_stride<N>() * 4;
  static constexpr size_t smem_z = (xz > fz ? xz : fz) + (size_t)NTW * 8;
  static constexpr int threads_z = 3 * LINES * P;
  // with the displacement fields: five pairs per line, half as many lines
  static constexpr int LINES_V = LINES >= 2 ? LINES / 2 : 1;
  static constexpr size_t xzv = (size_t)XLayoutLines<E, P, 5 * LINES_V, P1>::kSize * 8;
  static constexpr size_t fzv = (size_t)LINES_V * 10 * field_stride<N>() * 4;
  static constexpr size_t smem_zv = (xzv > fzv ? xzv : fzv) + (size_t)NTW * 8;
  static constexpr int threads_zv = 5 * LINES_V * P;
  // forward z: NCF complex transforms (two real lines each) per block
  static constexpr int NCF = P >= 64 ? 3 : 3 * (64 / P);
  static constexpr size_t xf = (size_t)XLayoutLines<E, P, NCF, P1>::kSize * 8;
  static constexpr size_t zf = (size_t)NCF * N * 8;
  static constexpr size_t smem_fz = (xf > zf ? xf : zf) + (size_t)NTW * 8;
};

// One x/y tile width: staged tile + exchange + twiddles + multipliers +
// alignment slack, and the block size.
template <int N, int TC> struct CfgXY {
  static constexpr int E = Shape<N>::E, P = Shape<N>::P, P1 = Shape<N>::P1, NTW = Shape<N>::kTw;
  static constexpr size_t smem = (size_t)N * TC * 8 + (size_t)XLayoutCols<E, P, TC, P1>::kSize * 8 +
                                 (size_t)NTW * 8 + (size_t)3 * N * 4 + 128;
  static constexpr int threads = TC * P;
};

// The x/y tile widths a plan may run (the autotuner's candidates): the
// default and half of it while a TMA box row stays at least 64 bytes.  Every
// width computes each column's transform with the same arithmetic, so the
// choice changes timings only.
template <int N> struct Tiles {
  static constexpr int T0 = Cfg<N>::TC;
  static constexpr int T1 = Cfg<N>::TC / 2 >= 8 ? Cfg<N>::TC / 2 : Cfg<N>::TC;
};

template <int N, int TC>
static cudaError_t set_attrs_xy() {
  constexpr int smem = (int)CfgXY<N, TC>::smem;
  cudaError_t e = cudaFuncSetAttribute(k_pass_x<N, TC>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_pass_y<N, TC, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_pass_y<N, TC, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

template <int N>
static cudaError_t set_attrs() {
  using C = Cfg<N>;
  cudaError_t e = set_attrs_xy<N, Tiles<N>::T0>();
  if (e != cudaSuccess) return e;
  if constexpr (Tiles<N>::T1 != Tiles<N>::T0) {
    e = set_attrs_xy<N, Tiles<N>::T1>();
    if (e != cudaSuccess) return e;
  }
  e = cudaFuncSetAttribute(k_pass_z<N, C::LINES, false, 3, C::FUSE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)C::smem_z);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_pass_z<N, C::LINES_V, false, 5, C::FUSE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)C::smem_zv);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_pass_z<N, C::LINES, false, 3, false, true>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem_z);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_fwd_z<N, C::NCF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem_fz);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_pass_z<N, C::LINES, true, 3, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)C::smem_z);
}

template <int N>
static PassShape shape_of() {
  using C = Cfg<N>;
  return PassShape{C::E, C::P, Shape<N>::P1, Shape<N>::P2, C::TC, C::LINES, CfgXY<N, C::TC>::smem, C::smem_z,
                   CfgXY<N, C::TC>::threads, C::threads_z};
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

template <int N, int TC>
static cudaError_t run_x(const ArgsX& a, cudaStream_t st) {
  using C = CfgXY<N, TC>;
  const long ntiles = (((long)a.ny * a.nhp + TC - 1) / TC) * a.batch;
  const unsigned grid = persistent_grid(k_pass_x<N, TC>, C::threads, C::smem, ntiles);
  k_pass_x<N, TC><<<grid, C::threads, C::smem, st>>>(a);
  return cudaGetLastError();
}

template <int N, int TC>
static cudaError_t run_y(const ArgsY& a, cudaStream_t st) {
  using C = CfgXY<N, TC>;
  const long ntiles = (long)a.nx * a.batch * ((a.nhp + TC - 1) / TC);
  bool dual = false;
  for (int o = 0; o < a.nout; ++o) dual = dual || a.dst2[o] != nullptr;
  if (dual) {
    const unsigned grid = persistent_grid(k_pass_y<N, TC, true>, C::threads, C::smem, ntiles);
    k_pass_y<N, TC, true><<<grid, C::threads, C::smem, st>>>(a);
  } else {
    const unsigned grid = persistent_grid(k_pass_y<N, TC, false>, C::threads, C::smem, ntiles);
    k_pass_y<N, TC, false><<<grid, C::threads, C::smem, st>>>(a);
  }
  return cudaGetLastError();
}

template <int N>
static cudaError_t run_z(const ArgsZ& a, bool dump, cudaStream_t st) {
  using C = Cfg<N>;
  const long nlines = a.nlines;
  if (!dump && a.nfields > 6) {
    const unsigned grid = (unsigned)((nlines + C::LINES_V - 1) / C::LINES_V);
    k_pass_z<N, C::LINES_V, false, 5, C::FUSE><<<grid, C::threads_zv, C::smem_zv, st>>>(a);
    return cudaGetLastError();
  }
  const unsigned grid = (unsigned)((nlines + C::LINES - 1) / C::LINES);
  if (dump) k_pass_z<N, C::LINES, true, 3, false><<<grid, C::threads_z, C::smem_z, st>>>(a);
  else k_pass_z<N, C::LINES, false, 3, C::FUSE><<<grid, C::threads_z, C::smem_z, st>>>(a);
  return cudaGetLastError();
}

template <int N>
static cudaError_t run_z_source(const ArgsZ& a, cudaStream_t st) {
  using C = Cfg<N>;
  const unsigned grid = (unsigned)((a.nlines + C::LINES - 1) / C::LINES);
  k_pass_z<N, C::LINES, false, 3, false, true><<<grid, C::threads_z, C::smem_z, st>>>(a);
  return cudaGetLastError();
}

template <int N>
static cudaError_t run_fwd_z(const float* src, float2* dst, int nlines, int nhp, const float2* tw,
                             cudaStream_t st) {
  using C = Cfg<N>;
  const int pairs = nlines / 2;
  const unsigned grid = (unsigned)((pairs + C::NCF - 1) / C::NCF);
  k_fwd_z<N, C::NCF><<<grid, C::NCF * C::P, C::smem_fz, st>>>(src, dst, nlines, nhp, tw);
  return cudaGetLastError();
}

#define PIN_SIZES(X) X(8) X(16) X(32) X(48) X(64) X(96) X(128) X(192) X(256) X(384) X(512) X(768)

bool z_fuses_roots(int n) {
  switch (n) {
#define CASE(N) case N: return Cfg<N>::FUSE;
    PIN_SIZES(CASE)
#undef CASE
    default: return false;
  }
}

bool size_supported(int n) {
  switch (n) {
#define CASE(N) case N: return true;
    PIN_SIZES(CASE)
#undef CASE
    default: return false;
  }
}

PassShape pass_shape(int n) {
  switch (n) {
#define CASE(N) case N: return shape_of<N>();
    PIN_SIZES(CASE)
#undef CASE
    default: return PassShape{};
  }
}

cudaError_t prepare_kernels(int n) {
  switch (n) {
#define CASE(N) case N: return set_attrs<N>();
    PIN_SIZES(CASE)
#undef CASE
    default: return cudaErrorInvalidValue;
  }
}

int xy_tile_options(int n, int* opts) {
  switch (n) {
#define CASE(N)                                             \
  case N:                                                   \
    opts[0] = Tiles<N>::T0;                                 \
    opts[1] = Tiles<N>::T1;                                 \
    return Tiles<N>::T1 != Tiles<N>::T0 ? 2 : 1;
    PIN_SIZES(CASE)
#undef CASE
    default: return 0;
  }
}

cudaError_t launch_x(int n, int tc, const ArgsX& a, cudaStream_t st) {
  switch (n) {
#define CASE(N) \
  case N: return tc == Tiles<N>::T1 ? run_x<N, Tiles<N>::T1>(a, st) : run_x<N, Tiles<N>::T0>(a, st);
    PIN_SIZES(CASE)
#undef CASE
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_y(int n, int tc, const ArgsY& a, cudaStream_t st) {
  switch (n) {
#define CASE(N) \
  case N: return tc == Tiles<N>::T1 ? run_y<N, Tiles<N>::T1>(a, st) : run_y<N, Tiles<N>::T0>(a, st);
    PIN_SIZES(CASE)
#undef CASE
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_z_source(int n, const ArgsZ& a, cudaStream_t st) {
  switch (n) {
#define CASE(N) case N: return run_z_source<N>(a, st);
    PIN_SIZES(CASE)
#undef CASE
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_fwd_z(int n, const float* src, float2* dst, int nlines, int nhp, const float2* tw,
                         cudaStream_t st) {
  if (nlines % 2) return cudaErrorInvalidValue;
  switch (n) {
#define CASE(N) case N: return run_fwd_z<N>(src, dst, nlines, nhp, tw, st);
    PIN_SIZES(CASE)
#undef CASE
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_phi2(const float2* T, float2* out, int nx, int ny, int nz, int nhp, double box, float scale,
                        cudaStream_t st) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  k_phi2<<<sms * 8, 256, 0, st>>>(T, out, nx, ny, nz, nhp, box, scale);
  return cudaGetLastError();
}

cudaError_t launch_z(int n, const ArgsZ& a, bool dump, cudaStream_t st) {
  switch (n) {
#define CASE(N) case N: return run_z<N>(a, dump, st);
    PIN_SIZES(CASE)
#undef CASE
    default: return cudaErrorInvalidValue;
  }
}

// ------------------------------------------------------------ tensor maps --

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                                   CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                   CUtensorMapFloatOOBfill);

static EncodeTiledFn tensor_map_encoder() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(ptr);
  });
  return fn;
}

// Complex64 elements are moved as 8-byte integers (no conversion; zero fill
// outside the tensor).
static cudaError_t encode(CUtensorMap* tm, int rank, const void* base, const cuuint64_t* dims,
                          const cuuint64_t* strides, const cuuint32_t* box) {
  EncodeTiledFn fn = tensor_map_encoder();
  if (!fn) return cudaErrorNotSupported;
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = fn(tm, CU_TENSOR_MAP_DATA_TYPE_INT64, (cuuint32_t)rank, const_cast<void*>(base), dims, strides,
                  box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t make_tmap_x(CUtensorMap* tm, const float2* src, int nx, int ny, int nhp, int batch, int tc) {
  const int boxes = (nx + 255) / 256;
  const cuuint64_t dims[2] = {(cuuint64_t)ny * nhp, (cuuint64_t)nx * batch};
  const cuuint64_t strides[1] = {(cuuint64_t)ny * nhp * 8};
  const cuuint32_t box[2] = {(cuuint32_t)tc, (cuuint32_t)(nx / boxes)};
  return encode(tm, 2, src, dims, strides, box);
}

cudaError_t make_tmap_y(CUtensorMap* tm, const float2* src3, int nx, int ny, int nhp, size_t spec_elems,
                        int batch, int tc) {
  const int boxes = (ny + 255) / 256;
  const cuuint64_t dims[4] = {(cuuint64_t)nhp, (cuuint64_t)ny, (cuuint64_t)nx * batch, 3};
  const cuuint64_t strides[3] = {(cuuint64_t)nhp * 8, (cuuint64_t)ny * nhp * 8, (cuuint64_t)spec_elems * 8};
  const cuuint32_t box[4] = {(cuuint32_t)tc, (cuuint32_t)(ny / boxes), 1, 1};
  return encode(tm, 4, src3, dims, strides, box);
}

cudaError_t upload_constant_twiddles() {
  float2 h[kTwTotal];
  for (int n : kTwSizes) {
    const int off = tw_offset(n);
    for (int j = 0; j < n; ++j) {
      const double ang = 2.0 * M_PI * (double)j / (double)n;
      h[off + j] = make_float2((float)std::cos(ang), (float)std::sin(ang));
    }
  }
  return cudaMemcpyToSymbol(c_tw, h, sizeof(h));
}

}  // namespace pin
