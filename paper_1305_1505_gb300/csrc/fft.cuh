// Register-resident inverse DFTs and the line FFTs (two or three levels) used
// by every pass of the collapse-time path: each smoothing radius needs the
// deformation tensor in real space, i.e. inverse 3D transforms of the
// filtered spectra (Sec. 2.1.1).
//
// Convention: inverse transforms, X[k] = sum_n x[n] exp(+2 pi i n k / N), no
// normalisation here (the 1/N of each axis is folded into the per-axis
// multiplier tables).
//
// Two-level decomposition of a length-N line, N = E * P:
//   n = p + P t   (p in [0,P): thread of the line, t in [0,E): register slot)
//   k = k1 + E k2 (k1 in [0,E), k2 in [0,P))
//   X[k1 + E k2] = sum_p w_P^{p k2} w_N^{p k1} sum_t w_E^{t k1} x[p + P t]
// Level 1 is a length-E DFT entirely in one thread's registers; after the
// twiddle w_N^{p k1} one shared-memory exchange hands every thread E/P values
// of k1 with all P values of p, and level 2 is E/P length-P DFTs, again in
// registers.  One shared-memory round trip per line and transform.
//
// Complex additions and the radix-2/3/4 butterflies use the packed FP32x2
// instructions (packed.cuh): the real and imaginary parts of a complex value
// are the two lanes of one register pair, and the multiplications by i in the
// radix-3 and radix-4 butterflies become a lane swap and one packed fma with
// a (-s, s) constant.
#pragma once
#include <cuda_runtime.h>

#include "packed.cuh"

namespace pin {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return x2::add(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return x2::sub(a, b); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cmuli(float2 a) { return make_float2(-a.y, a.x); }  // a * i
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }

// exp(+2 pi i j / n) for the register-DFT sizes, filled once per device from
// double precision host values.  Indices are compile-time constants after
// unrolling, so every read is a constant-bank operand.
constexpr int kTwSizes[] = {4, 8, 12, 16, 24, 32, 48, 64};
constexpr int kTwTotal = 4 + 8 + 12 + 16 + 24 + 32 + 48 + 64;
__host__ __device__ constexpr int tw_offset(int n) {
  return n == 4 ? 0 : n == 8 ? 4 : n == 12 ? 12 : n == 16 ? 24 : n == 24 ? 40
       : n == 32 ? 64 : n == 48 ? 96 : n == 64 ? 144 : -1;
}
// Defined here: every translation unit that includes this header has a copy
// of its own (separate device code), which that unit fills with
// upload_tw_table_here (kernels.cu and kernels_v1.cu, through
// upload_constant_twiddles).
__constant__ float2 c_tw[kTwTotal];

static inline cudaError_t upload_tw_table_here() {
  float2 h[kTwTotal];
  for (int n : kTwSizes) {
    const int off = tw_offset(n);
    for (int j = 0; j < n; ++j) {
      const double ang = 2.0 * 3.14159265358979323846 * (double)j / (double)n;
      h[off + j] = make_float2((float)cos(ang), (float)sin(ang));
    }
  }
  return cudaMemcpyToSymbol(c_tw, h, sizeof(h));
}

template <int N>
__device__ __forceinline__ float2 twc(int j) {
  static_assert(tw_offset(N) >= 0, "no twiddle table for this size");
  return c_tw[tw_offset(N) + j];
}

template <int N> struct DFT;

template <> struct DFT<1> {
  __device__ __forceinline__ static void run(float2 (&)[1]) {}
};

template <> struct DFT<2> {
  __device__ __forceinline__ static void run(float2 (&v)[2]) {
    float2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  }
};

template <> struct DFT<3> {
  __device__ __forceinline__ static void run(float2 (&v)[3]) {
    // w = exp(2 pi i / 3) = -1/2 + i sqrt(3)/2:
    // X1 = m + i h d, X2 = m - i h d with m = a - s/2, s = v1 + v2, d = v1 - v2,
    // and i h d = swap(d) * (-h, h)
    const float h = 0.86602540378443864676f;
    const float2 a = v[0], s = cadd(v[1], v[2]), ds = x2::swap(csub(v[1], v[2]));
    const float2 m = x2::fma(s, x2::splat(-0.5f), a);
    v[0] = cadd(a, s);
    v[1] = x2::fma(ds, make_float2(-h, h), m);
    v[2] = x2::fma(ds, make_float2(h, -h), m);
  }
};

template <> struct DFT<4> {
  __device__ __forceinline__ static void run(float2 (&v)[4]) {
    // X1 = d02 + i t, X3 = d02 - i t with t = v1 - v3, i t = swap(t) * (-1, 1)
    const float2 s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
    const float2 s13 = cadd(v[1], v[3]), ts = x2::swap(csub(v[1], v[3]));
    v[0] = cadd(s02, s13);
    v[2] = csub(s02, s13);
    v[1] = x2::fma(ts, make_float2(-1.f, 1.f), d02);
    v[3] = x2::fma(ts, make_float2(1.f, -1.f), d02);
  }
};

// Composite N = R * M, natural order in and out:
//   n = M r + m, k = k1 + R k2:  X[k1 + R k2] = sum_m w_M^{m k2} w_N^{m k1} DFT_R(x[M r + m])[k1]
template <int R, int M>
__device__ __forceinline__ void dft_split(float2 (&v)[R * M]) {
  constexpr int N = R * M;
  float2 y[N];
#pragma unroll
  for (int m = 0; m < M; ++m) {
    float2 t[R];
#pragma unroll
    for (int r = 0; r < R; ++r) t[r] = v[M * r + m];
    DFT<R>::run(t);
#pragma unroll
    for (int k1 = 0; k1 < R; ++k1) y[M * k1 + m] = (m * k1 == 0) ? t[k1] : cmul(t[k1], twc<N>(m * k1));
  }
#pragma unroll
  for (int k1 = 0; k1 < R; ++k1) {
    float2 t[M];
#pragma unroll
    for (int m = 0; m < M; ++m) t[m] = y[M * k1 + m];
    DFT<M>::run(t);
#pragma unroll
    for (int k2 = 0; k2 < M; ++k2) v[k1 + R * k2] = t[k2];
  }
}

template <int N> struct SplitOf;
template <> struct SplitOf<8> { static constexpr int R = 2; };
template <> struct SplitOf<12> { static constexpr int R = 3; };
template <> struct SplitOf<16> { static constexpr int R = 4; };
template <> struct SplitOf<24> { static constexpr int R = 3; };
template <> struct SplitOf<32> { static constexpr int R = 4; };
template <> struct SplitOf<48> { static constexpr int R = 3; };
template <> struct SplitOf<64> { static constexpr int R = 4; };

template <int N> struct DFT {
  __device__ __forceinline__ static void run(float2 (&v)[N]) {
    dft_split<SplitOf<N>::R, N / SplitOf<N>::R>(v);
  }
};

// Per-size decomposition N = E * P of a line (E register slots per thread,
// P threads per line).  Two levels (P2 == 1): P divides E, so that level 2
// hands each thread E/P whole length-P transforms.  Three levels (P2 > 1,
// P = P1 * P2): the length-P transforms are themselves split into a length-P2
// stage and a length-P1 stage with a second exchange, so that E, and with it
// the registers a thread holds, stays small (P1 and P2 divide E).
// Each size has two radix schedules: V = 0 (the default of every pass) and
// V = 1, another split of the same length that the x and y passes can run
// (pin_autotune times both); the z pass always runs V = 0.
template <int N, int V = 0> struct ShapeBase;
template <> struct ShapeBase<8, 0>    { static constexpr int E = 8,  P1 = 1, P2 = 1; };
template <> struct ShapeBase<16, 0>   { static constexpr int E = 16, P1 = 1, P2 = 1; };
template <> struct ShapeBase<32, 0>   { static constexpr int E = 8,  P1 = 4, P2 = 1; };
template <> struct ShapeBase<48, 0>   { static constexpr int E = 12, P1 = 4, P2 = 1; };
template <> struct ShapeBase<64, 0>   { static constexpr int E = 8,  P1 = 8, P2 = 1; };
template <> struct ShapeBase<96, 0>   { static constexpr int E = 24, P1 = 4, P2 = 1; };
template <> struct ShapeBase<128, 0>  { static constexpr int E = 16, P1 = 8, P2 = 1; };
template <> struct ShapeBase<192, 0>  { static constexpr int E = 24, P1 = 8, P2 = 1; };
template <> struct ShapeBase<256, 0>  { static constexpr int E = 16, P1 = 16, P2 = 1; };
#ifndef PIN_384_TWO_LEVEL
template <> struct ShapeBase<384, 0>  { static constexpr int E = 24, P1 = 4, P2 = 4; };
#else
template <> struct ShapeBase<384, 0>  { static constexpr int E = 48, P1 = 8, P2 = 1; };
#endif
template <> struct ShapeBase<512, 0>  { static constexpr int E = 32, P1 = 16, P2 = 1; };
#ifndef PIN_768_TWO_LEVEL
template <> struct ShapeBase<768, 0>  { static constexpr int E = 24, P1 = 4, P2 = 8; };
#else
template <> struct ShapeBase<768, 0>  { static constexpr int E = 48, P1 = 16, P2 = 1; };
#endif
// the alternative schedules
template <> struct ShapeBase<8, 1>    { static constexpr int E = 4,  P1 = 2, P2 = 1; };
template <> struct ShapeBase<16, 1>   { static constexpr int E = 4,  P1 = 4, P2 = 1; };
template <> struct ShapeBase<32, 1>   { static constexpr int E = 16, P1 = 2, P2 = 1; };
template <> struct ShapeBase<48, 1>   { static constexpr int E = 24, P1 = 2, P2 = 1; };
template <> struct ShapeBase<64, 1>   { static constexpr int E = 16, P1 = 4, P2 = 1; };
template <> struct ShapeBase<96, 1>   { static constexpr int E = 12, P1 = 4, P2 = 2; };
template <> struct ShapeBase<128, 1>  { static constexpr int E = 8,  P1 = 4, P2 = 4; };
template <> struct ShapeBase<192, 1>  { static constexpr int E = 12, P1 = 4, P2 = 4; };
template <> struct ShapeBase<256, 1>  { static constexpr int E = 16, P1 = 4, P2 = 4; };
template <> struct ShapeBase<384, 1>  { static constexpr int E = 24, P1 = 8, P2 = 2; };
template <> struct ShapeBase<512, 1>  { static constexpr int E = 32, P1 = 4, P2 = 4; };
template <> struct ShapeBase<768, 1>  { static constexpr int E = 24, P1 = 8, P2 = 4; };
template <int N, int V = 0> struct Shape : ShapeBase<N, V> {
  static constexpr int E = ShapeBase<N, V>::E, P1 = ShapeBase<N, V>::P1, P2 = ShapeBase<N, V>::P2;
  static constexpr int P = P1 * P2;
  // twiddles: w_N^{p k1} ([k1][p], E*P = N entries), then for three levels
  // w_P^{p1 k2a} ([k2a][p1], P entries)
  static constexpr int kTw = E * P + (P2 > 1 ? P : 0);
  static_assert(E * P == N, "shape must cover the line");
  static_assert(E % P1 == 0 && E % P2 == 0, "stage lengths must divide E");
};

// Shared-memory layouts for the level-1 -> level-2 exchange of one tile of
// lines.  Index of value (k1, p) of line c.
//  - Strided lines (passes along x and y): consecutive lanes are consecutive
//    lines (columns of a row-major array), layout [k1][p][c].
//  - Contiguous lines (pass along z): consecutive lanes are consecutive p of
//    one line, layout [c][k1][p] with the p extent padded to P+1 so that the
//    level-2 reads (stride P+1) do not collide on a bank.
// at(k1, p, c): exchange after level 1; at2(k1, k2a, p1, c): second exchange
// of the three-level form (P = P1 P2).
// In at2 the p1 index is flipped in its lowest bit for odd k2a: a level-3
// read (lanes over consecutive k2a and the columns) then alternates between
// bank halves when the columns fill only half of the banks (TC = 8); for
// wider tiles it is a harmless permutation within each row.
template <int E, int P, int TC, int P1 = P>
struct XLayoutCols {
  static constexpr int P2 = P / P1;
  static constexpr int kSize = E * P * TC;
  __device__ __forceinline__ static int at(int k1, int p, int c) { return (k1 * P + p) * TC + c; }
  __device__ __forceinline__ static int at2(int k1, int k2a, int p1, int c) {
    if constexpr (P1 > 1) p1 ^= (k2a & 1);
    return ((k1 * P2 + k2a) * P1 + p1) * TC + c;
  }
};
template <int E, int P, int NC, int P1 = P>
struct XLayoutLines {
  static constexpr int P2 = P / P1;
  // two levels: per-line stride padded to P (mod 16) float2, so that the 32/P
  // lines of a warp (each 2P banks wide) tile the 32 banks
  static constexpr int kLine0 = E * (P + 1);
  static constexpr int kLine2 = P >= 16 ? kLine0 : kLine0 + ((P - kLine0 % 16) % 16 + 16) % 16;
  // three levels (one line per warp, lanes p = p1 + P1 q): rows of the first
  // exchange are S1 >= P float2 with S1 = P1 (mod 16), so lanes (q, p1) of a
  // level-2 read spread over the banks; the second exchange is [k2a][k1][p1]
  // with a row of S2 = 1 (mod 16) float2 per k2a, so both its writes (lanes
  // (q, p1)) and its level-3 reads (lanes (k1, k2a)) spread too.
  static constexpr int S1 = P + ((P1 - P % 16) % 16 + 16) % 16;
  static constexpr int S2 = E * P1 + ((1 - (E * P1) % 16) % 16 + 16) % 16;
  static constexpr int kLine3 = (E * S1 > P2 * S2) ? E * S1 : P2 * S2;
  static constexpr int kLine = P2 > 1 ? kLine3 : kLine2;
  static constexpr int kSize = NC * kLine;
  __device__ __forceinline__ static int at(int k1, int p, int c) {
    if constexpr (P2 > 1) return c * kLine + k1 * S1 + p;
    else return c * kLine + k1 * (P + 1) + p;
  }
  __device__ __forceinline__ static int at2(int k1, int k2a, int p1, int c) {
    return c * kLine + k2a * S2 + k1 * P1 + p1;
  }
};

// A twiddle: from shared memory, or (TWG) from the global table through the
// read-only cache.
template <bool TWG>
__device__ __forceinline__ float2 ld_tw(const float2* tw) {
  if constexpr (TWG) return __ldg(tw);
  else return *tw;
}
// Level-2 twiddles w_N^{p k1}, laid out [k1][p].
template <int E, int P, bool TWG = false>
__device__ __forceinline__ float2 tw2(const float2* s_tw, int k1, int p) { return ld_tw<TWG>(s_tw + k1 * P + p); }

// Inverse FFT of one line held as v[t] = x[p + P t] by thread p of the line.
// Two levels: on return v[i * P + k2] = X[(p + P i) + E k2] for i in [0, E/P),
// k2 in [0, P) (for P == 1: v[k] = X[k]).  Three levels (P = P1 P2, with
// p = p1 + P1 q): X[k1 + E (k2a + P2 k2b)] = sum_p1 w_P1^{p1 k2b} w_P^{p1 k2a}
// sum_p2 w_P2^{p2 k2a} w_N^{p k1} Y_p[k1], Y_p the level-1 DFT of thread p;
// on return v[m P1 + k2b] holds the pair (k1, k2a) = divmod(p + P m, P2).
// fft_out_index gives the frequency of each slot.  All threads of the block
// must call it; it synchronises once (twice more for three levels) and leaves
// the exchange buffer in use (callers synchronise the block before writing
// s_x again).  WARP: every transform is held within one warp (P divides 32,
// transform c on threads [c P, c P + P)) with an exchange region of its own,
// so those synchronisations are warp-level.  TWG: s_tw is the global twiddle
// table (same layout), read through the read-only cache.
// No-op hook for fft_line.
struct NoHook {
  __device__ __forceinline__ void operator()() const {}
};
template <int N, class Layout, bool WARP = false, int V = 0, bool TWG = false, class Hook = NoHook>
__device__ __forceinline__ void fft_line(float2 (&v)[Shape<N, V>::E], int p, int c, float2* s_x,
                                         const float2* s_tw, Hook before_exchange = Hook()) {
  using S = Shape<N, V>;
  constexpr int E = S::E, P = S::P, P1 = S::P1, P2 = S::P2;
  static_assert(!WARP || 32 % P == 0, "warp-level exchanges need whole transforms per warp");
  auto sync = [] {
    if constexpr (WARP) __syncwarp();
    else __syncthreads();
  };
  DFT<E>::run(v);
  before_exchange();  // all threads of the block: nothing has touched s_x yet
  if constexpr (P2 > 1) {
    // level 1 done; twiddle w_N^{p k1} and first exchange
#pragma unroll
    for (int k1 = 0; k1 < E; ++k1) {
      float2 z = (k1 == 0) ? v[k1] : cmul(v[k1], tw2<E, P, TWG>(s_tw, k1, p));
      s_x[Layout::at(k1, p, c)] = z;
    }
    sync();
    // level 2: for k1 = q + P2 i, the length-P2 DFT over p2 of Z[k1][p1 + P1 p2],
    // then the twiddle w_P^{p1 k2a}
    const int p1 = p % P1, q = p / P1;
    float2 twb[P2];  // w_P^{p1 k2a}: the same for every k1 of this thread
#pragma unroll
    for (int k2a = 1; k2a < P2; ++k2a) twb[k2a] = ld_tw<TWG>(s_tw + E * P + k2a * P1 + p1);
#pragma unroll
    for (int i = 0; i < E / P2; ++i) {
      float2 t[P2];
#pragma unroll
      for (int j = 0; j < P2; ++j) t[j] = s_x[Layout::at(q + P2 * i, p1 + P1 * j, c)];
      DFT<P2>::run(t);
#pragma unroll
      for (int k2a = 0; k2a < P2; ++k2a) v[i * P2 + k2a] = (k2a == 0) ? t[k2a] : cmul(t[k2a], twb[k2a]);
    }
    sync();
#pragma unroll
    for (int i = 0; i < E / P2; ++i)
#pragma unroll
      for (int k2a = 0; k2a < P2; ++k2a) s_x[Layout::at2(q + P2 * i, k2a, p1, c)] = v[i * P2 + k2a];
    sync();
    // level 3: pairs (k1, k2a) = divmod(p + P m, P2), the length-P1 DFT over p1
#pragma unroll
    for (int m = 0; m < E / P1; ++m) {
      const int pi = p + P * m;
      const int k1 = pi / P2, k2a = pi % P2;
      float2 t[P1];
#pragma unroll
      for (int r = 0; r < P1; ++r) t[r] = s_x[Layout::at2(k1, k2a, r, c)];
      DFT<P1>::run(t);
#pragma unroll
      for (int k2b = 0; k2b < P1; ++k2b) v[m * P1 + k2b] = t[k2b];
    }
  } else if constexpr (P > 1) {
#pragma unroll
    for (int k1 = 0; k1 < E; ++k1) {
      float2 z = (k1 == 0) ? v[k1] : cmul(v[k1], tw2<E, P, TWG>(s_tw, k1, p));
      s_x[Layout::at(k1, p, c)] = z;
    }
    sync();
#pragma unroll
    for (int i = 0; i < E / P; ++i) {
      float2 t[P];
#pragma unroll
      for (int q = 0; q < P; ++q) t[q] = s_x[Layout::at(p + P * i, q, c)];
      DFT<P>::run(t);
#pragma unroll
      for (int k2 = 0; k2 < P; ++k2) v[i * P + k2] = t[k2];
    }
  } else {
    (void)p; (void)c; (void)s_x; (void)s_tw;
  }
}

// Output frequency of register slot j after fft_line.
template <int N, int V = 0>
__device__ __forceinline__ int fft_out_index(int p, int j) {
  using S = Shape<N, V>;
  constexpr int E = S::E, P = S::P, P1 = S::P1, P2 = S::P2;
  if constexpr (P2 > 1) {
    const int m = j / P1, k2b = j % P1;
    const int pi = p + P * m;
    return pi / P2 + E * (pi % P2 + P2 * k2b);
  } else if constexpr (P == 1) {
    (void)p;
    return j;
  } else {
    int i = j / P, k2 = j % P;
    return p + P * i + E * k2;
  }
}

}  // namespace pin
