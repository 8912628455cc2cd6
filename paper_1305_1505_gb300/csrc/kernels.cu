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
#include "passes_xy.cuh"

namespace pin {

// Stride (floats) of one real field line in the z pass's shared buffer, padded
// so that the stores of the transform outputs spread over the banks: two-level
// lines write runs of P consecutive z per pair-column (offset P/2), three-level
// lines write z = k1 + E (k2a + P2 k2b) (offset 2, so that the two
// pair-columns of a 16-thread-line warp land on disjoint banks).
template <int N> __host__ __device__ constexpr int field_stride() {
  return Shape<N>::P2 > 1 ? N + 2 : N + (Shape<N>::P >= 2 ? Shape<N>::P / 2 : 1);
}

// Compaction of the root solve in the fused z pass (1: queue the particles
// that cannot be skipped and solve them after the main loop).
#ifndef PIN_Z_COMPACT
#define PIN_Z_COMPACT 1
#endif

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
__global__ void __launch_bounds__(NP * LINES * Shape<N>::P, NP == 5 ? MinBlocks<N>::zv : MinBlocks<N>::z)
    k_pass_z(ArgsZ a) {
  constexpr int E = Shape<N>::E, P = Shape<N>::P;
  constexpr int NC = NP * LINES;  // pair-columns of the block
  constexpr int NF = 2 * NP;      // field slots per line
  using L = XLayoutLines<E, P, NC, Shape<N>::P1>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float2* s_x = reinterpret_cast<float2*>(smem_raw);
  constexpr int kFS = field_stride<N>();
  float* s_f = reinterpret_cast<float*>(smem_raw);
  __shared__ int s_nq;  // queued particles (compaction of the root solve)
  const int nthreads = NC * P;
  const int tid = threadIdx.x;
  // the lines of the block that starts about one wave of resident blocks
  // later go to L2 now (one bulk prefetch per field), so that its first
  // loads wait on L2 rather than on DRAM
  if (a.prefetch_blocks > 0 && tid < a.nfields) {
    const long long ahead = (long long)(blockIdx.x + a.prefetch_blocks) * LINES;
    if (ahead + LINES <= a.nlines) {
      const float2* ptr = a.src[tid] + (size_t)ahead * a.nhp;
      const unsigned bytes = (unsigned)(LINES * a.nhp * sizeof(float2));  // nhp % 4 == 0: a multiple of 32
      asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(ptr), "r"(bytes) : "memory");
    }
  }

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
  if constexpr (Shape<N>::P2 > 1) {
    // three-level lines: twiddles from the global table through the
    // read-only cache (a few KB, cached for every block on the SM), so that a
    // block starts with its spectrum loads instead of a copy and a barrier
    // (z pass 5.87 -> 5.52 ms per radius at 768^3)
    fft_line<N, L, 32 % Shape<N>::P == 0, 0, true>(v, p, c, s_x, a.tw);
  } else {
    // two-level lines: a shared-memory copy behind the field buffer, made
    // after the spectrum loads are issued (256^3: 0.18 -> 0.16 ms per radius
    // against the read-only cache)
    constexpr int kXB = L::kSize * 8, kFB = LINES * NF * kFS * 4 + LINES * N * 2;
    float2* s_tw = reinterpret_cast<float2*>(smem_raw + (kXB > kFB ? kXB : kFB));
    for (int i = tid; i < Shape<N>::kTw; i += nthreads) s_tw[i] = a.tw[i];
    __syncthreads();
    fft_line<N, L, 32 % Shape<N>::P == 0>(v, p, c, s_x, s_tw);
  }

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
    constexpr int kPts = LINES * N;
    if (tid == 0) s_nq = 0;
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
      // Compaction: particles that cannot be skipped are queued and solved
      // after the main loop, two per thread, so that a warp's root solve runs
      // on full lanes
      constexpr bool kCompact = PIN_Z_COMPACT != 0;
      unsigned short* s_q = reinterpret_cast<unsigned short*>(s_f + LINES * NF * kFS);
      // The end of a pair's computation: the rare minor-axis solve, the FP64
      // redo of an ill-conditioned root, and the running maximum.
      auto finish = [&](CollapseStateX2& cx, unsigned dn, const float2 (&lm)[3], const int (&qv)[2],
                        const int (&lzv)[2], const float (&fmv)[2]) {
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          if ((dn >> u) & 1u) continue;
          CollapseState<float> cs = lane_state(cx, u);
          if (cs.need[0] || cs.need[1]) collapse_rare<float>(cs);
          const int qq = qv[u];
          const float F = cs.best + cs.corr;
          if (cs.kappa < a.tau_root) {
            atomicAdd(a.counters + 1, 1ull);
            const unsigned slot = atomicAdd(a.redo_count, 1u);
            if (slot < a.redo_cap) {
              RedoEntry e;
              e.q = qq;
#pragma unroll
              for (int k = 0; k < 3; ++k) e.h[k] = u ? lm[k].y : lm[k].x;
              e.h[3] = e.h[4] = e.h[5] = 0.f;
              e.kind = 1;
              a.redo_list[slot] = e;
              if constexpr (NP == 5) {
#pragma unroll
                for (int cpt = 0; cpt < 3; ++cpt) a.psi_out[cpt * total + qq] = s_f[lzv[u] + (6 + cpt) * kFS];
              }
              continue;
            }
            atomicAdd(a.counters + 2, 1ull);  // queue full: keep the FP32 value
          }
          if (F > fmv[u] || (F == fmv[u] && F > 0.f && a.scale < a.idx[qq])) {
            a.fmax[qq] = F;
            a.idx[qq] = a.scale;
            if constexpr (NP == 5) {
#pragma unroll
              for (int cpt = 0; cpt < 3; ++cpt) a.vstate[cpt * total + qq] = s_f[lzv[u] + (6 + cpt) * kFS];
            }
          }
        }
      };
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
              // a near-degenerate pair: the FP32 eigenvalues are not trusted,
              // but the invariant bound (no eigenvalues) may already show that
              // the particle cannot beat F_max, by more than the FP32 error of
              // the bound; then neither the redo nor anything else is needed
              float hl[6];
#pragma unroll
              for (int f = 0; f < 6; ++f) hl[f] = u ? h[f].y : h[f].x;
              if (fm[r][u] * (1.f - 1e-5f) > collapse_bound<float>(hl, ccf) * (1.f + 1e-5f)) {
                valid[r][u] = false;
                continue;
              }
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
        // FP64 redo finishes skip the root solve
        CollapseStateX2 csx[NPR];
        unsigned done[NPR];
#pragma unroll
        for (int r = 0; r < NPR; ++r) {
          float2 c0[3];
          collapse_prep_x2(lam[r], ccf, csx[r], c0);
          done[r] = cannot_beat_x2(c0, csx[r], make_float2(fm[r][0], fm[r][1])) | (valid[r][0] ? 0u : 1u) |
                    (valid[r][1] ? 0u : 2u);
          if constexpr (kCompact) {
            // the rest wait in a queue: eigenvalues and F_max in the
            // particle's own (already read) field slots 0-3
#pragma unroll
            for (int u = 0; u < 2; ++u) {
              if ((done[r] >> u) & 1u) continue;
#pragma unroll
              for (int k = 0; k < 3; ++k) s_f[lz[r][u] + k * kFS] = u ? lam[r][k].y : lam[r][k].x;
              s_f[lz[r][u] + 3 * kFS] = fm[r][u];
              s_q[atomicAdd(&s_nq, 1)] = (unsigned short)(pt0 + (2 * r + u) * nthreads);
            }
          } else {
            // a pair solves if one of its lanes needs it
            if (done[r] != 3u) collapse_root_x2(c0, csx[r]);
          }
        }
        if constexpr (!kCompact) {
#pragma unroll
          for (int r = 0; r < NPR; ++r) finish(csx[r], done[r], lam[r], q[r], lz[r], fm[r]);
        }
      }
      if constexpr (kCompact) {
        // the queued particles, two per thread: the lanes of a warp all need
        // the root (in the main loop a warp solved whenever one of its 64
        // particles did: about 40 % of warps for 7 % of pairs at 768^3; z
        // pass 5.52 -> 5.21 ms per radius)
        __syncthreads();
        const int nq = s_nq;
        for (int k0 = 2 * tid; k0 < nq; k0 += 2 * nthreads) {
          int q2[2], lz2[2];
          float fm2[2];
          float2 lam2[3];
          unsigned dn = 0;
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const bool ok = k0 + u < nq;
            const int pt = s_q[ok ? k0 + u : k0];
            const int l = pt / N, z = pt % N;
            q2[u] = (blockIdx.x * LINES + l) * N + z;
            lz2[u] = (l * NF) * kFS + z;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
              const float x = s_f[lz2[u] + k * kFS];
              if (u) lam2[k].y = x;
              else lam2[k].x = x;
            }
            fm2[u] = s_f[lz2[u] + 3 * kFS];
            dn |= ok ? 0u : (1u << u);
          }
          CollapseStateX2 cs2;
          float2 c0[3];
          collapse_prep_x2(lam2, ccf, cs2, c0);
          collapse_root_x2(c0, cs2);
          finish(cs2, dn, lam2, q2, lz2, fm2);
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
    // the invariant bound (the six components, or diag(lambda) for kind 1)
    // first: below F_max by more than the FP32 rounding of F, the particle
    // cannot be updated, and the FP64 eigenvalues and roots are skipped
    const float fm0 = a.fmax[e.q];
    if ((double)fm0 * (1.0 - 1e-6) > collapse_bound<double>(h, ccd)) continue;
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
  // z-pass lines per block: 64 threads' worth of line per pair (at the
  // three-level sizes one 32-thread line: 768 -> 1, 384 -> 2)
#ifndef PIN_Z_LW3
#define PIN_Z_LW3 32
#endif
  static constexpr int LINES = P >= 64 ? 1 : (Shape<N>::P2 > 1 ? PIN_Z_LW3 : 64) / P;
  // the root solve runs inside the z pass where its transform leaves the
  // registers for it (three-level lines)
#ifndef PIN_Z_FUSE
  static constexpr bool FUSE = Shape<N>::P2 > 1;
#else
  static constexpr bool FUSE = PIN_Z_FUSE != 0;
#endif
  static constexpr size_t xz = (size_t)XLayoutLines<E, P, 3 * LINES, P1>::kSize * 8;
  static constexpr size_t fz = (size_t)LINES * 6 * field_stride<N>() * 4;
  // the field buffer is followed by the queue of the root solve (one 16-bit
  // index per particle); twiddles come through the read-only cache
  static constexpr size_t fzq = fz + (size_t)LINES * N * 2;
  static constexpr size_t tw_z = Shape<N>::P2 > 1 ? 0 : (size_t)NTW * 8;  // two-level: twiddle copy
  static constexpr size_t smem_z = (xz > fzq ? xz : fzq) + tw_z;
  static constexpr int threads_z = 3 * LINES * P;
  // with the displacement fields: five pairs per line, half as many lines
  static constexpr int LINES_V = P >= 64 ? 1 : (64 / P >= 2 ? 64 / P / 2 : 1);
  static constexpr size_t xzv = (size_t)XLayoutLines<E, P, 5 * LINES_V, P1>::kSize * 8;
  static constexpr size_t fzv = (size_t)LINES_V * 10 * field_stride<N>() * 4;
  static constexpr size_t fzvq = fzv + (size_t)LINES_V * N * 2;
  static constexpr size_t smem_zv = (xzv > fzvq ? xzv : fzvq) + tw_z;
  static constexpr int threads_zv = 5 * LINES_V * P;
  // forward z: NCF complex transforms (two real lines each) per block
  static constexpr int NCF = P >= 64 ? 3 : 3 * (64 / P);
  static constexpr size_t xf = (size_t)XLayoutLines<E, P, NCF, P1>::kSize * 8;
  static constexpr size_t zf = (size_t)NCF * N * 8;
  static constexpr size_t smem_fz = (xf > zf ? xf : zf) + (size_t)NTW * 8;
};

template <int N>
static cudaError_t set_attrs() {
  using C = Cfg<N>;
  cudaError_t e = set_attrs_xy_all<N, 0>();
  if (e != cudaSuccess) return e;
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
  return PassShape{C::E, C::P, Shape<N>::P1, Shape<N>::P2, C::TC, C::LINES, CfgXY<N, C::TC, 0>::smem, C::smem_z,
                   CfgXY<N, C::TC, 0>::threads, C::threads_z};
}

// Blocks of a z-pass launch resident on the device at once: the distance of
// its L2 prefetch.
template <class K>
static int resident_blocks(K kernel, int threads, size_t smem) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
  return std::max(1, sms) * std::max(1, per_sm);
}

template <int N>
static cudaError_t run_z(const ArgsZ& a_in, bool dump, cudaStream_t st) {
  using C = Cfg<N>;
  ArgsZ a = a_in;
  const long nlines = a.nlines;
  // one wave ahead: measured best against none and two waves (384^3 z pass
  // 0.80 -> 0.76 ms, 768^3 5.93 -> 5.89 ms per radius)
  static const int wave = resident_blocks(k_pass_z<N, C::LINES, false, 3, C::FUSE>, C::threads_z, C::smem_z);
  if (!dump && a.nfields <= 6) a.prefetch_blocks = wave;
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
  cudaError_t e = cudaErrorInvalidValue;
  switch (n) {
#define CASE(N) case N: e = set_attrs<N>(); break;
    PIN_SIZES(CASE)
#undef CASE
    default: return cudaErrorInvalidValue;
  }
  return e == cudaSuccess ? prepare_xy_v1(n) : e;
}

int xy_tile_options(int n, int v, int* opts) {
  if (v == 1) return xy_tile_options_v1(n, opts);
  if (v != 0) return 0;
  switch (n) {
#define CASE(N)                                             \
  case N:                                                   \
    opts[0] = Tiles<N, 0>::T0;                              \
    opts[1] = Tiles<N, 0>::T1;                              \
    return Tiles<N, 0>::T1 != Tiles<N, 0>::T0 ? 2 : 1;
    PIN_SIZES(CASE)
#undef CASE
    default: return 0;
  }
}

PassShape pass_shape_xy(int n, int v) {
  if (v == 1) return pass_shape_xy_v1(n);
  switch (n) {
#define CASE(N) case N: return xy_shape_of<N, 0>();
    PIN_SIZES(CASE)
#undef CASE
    default: return PassShape{};
  }
}

cudaError_t launch_x(int n, int tc, int v, const ArgsX& a, cudaStream_t st) {
  if (v == 1) return launch_x_v1(n, tc, a, st);
  switch (n) {
#define CASE(N) case N: return launch_x_v<N, 0>(tc, a, st);
    PIN_SIZES(CASE)
#undef CASE
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_y(int n, int tc, int v, const ArgsY& a, cudaStream_t st) {
  if (v == 1) return launch_y_v1(n, tc, a, st);
  switch (n) {
#define CASE(N) case N: return launch_y_v<N, 0>(tc, a, st);
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

cudaError_t make_tmap_rows(CUtensorMap* tm, const float2* base, int cols, long long rows, int tc, int box_rows) {
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)cols * 8};
  const cuuint32_t box[2] = {(cuuint32_t)tc, (cuuint32_t)box_rows};
  return encode(tm, 2, base, dims, strides, box);
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
  const cudaError_t e = upload_tw_table_here();
  return e == cudaSuccess ? upload_constant_twiddles_v1() : e;
}

}  // namespace pin
