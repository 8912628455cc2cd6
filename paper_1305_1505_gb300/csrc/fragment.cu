// Fragmentation front end (Sec. 2.1.2): the order in which the particles are
// considered (descending F_max; ties by ascending particle index, a reading:
// the paper gives no tie rule) and, per particle, how many of its six grid
// neighbours come before it in that order (0: the particle is a peak of the
// F_max field and starts a new halo, case (i); the sequential accretion and
// merging that follow stay with the caller).
//
// The order is a stable least-significant-digit radix sort of the keys
// ~bits(F_max) (F_max >= 0 and never NaN, so the unsigned order of the keys is
// the descending order of F) carrying the particle index: four passes of
// 8 bits, each a tile histogram, an exclusive scan of the digit-major
// histogram table, and a scatter that ranks each tile in shared memory and
// writes runs of equal digits to consecutive addresses.  Pass 0 reads F_max
// directly and makes the index on the fly; the last pass writes only the
// indices.
#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.cuh"

namespace pin {
namespace {

constexpr int kThreads = 256;
constexpr int kItems = 16;
constexpr int kTile = kThreads * kItems;  // keys per block
constexpr int kWarps = kThreads / 32;
constexpr int kBins = 256;

__device__ __forceinline__ uint32_t fkey(float f) { return ~__float_as_uint(f); }

template <bool FIRST>
__global__ void __launch_bounds__(kThreads) k_rs_hist(const uint32_t* __restrict__ keys,
                                                      const float* __restrict__ fmax, long n, int shift,
                                                      uint32_t* hist, int ntiles) {
  __shared__ uint32_t s_h[kBins];
  const int tid = threadIdx.x;
  s_h[tid] = 0;
  __syncthreads();
  const long base = (long)blockIdx.x * kTile;
  // plain shared-memory atomics: measured as fast as warp-aggregated ones on
  // the clustered top byte, and much faster on the spread low bytes
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    const long idx = base + (long)i * kThreads + tid;
    if (idx < n) {
      const uint32_t k = FIRST ? fkey(__ldg(fmax + idx)) : __ldg(keys + idx);
      atomicAdd(&s_h[(k >> shift) & 255u], 1u);
    }
  }
  __syncthreads();
  hist[(size_t)tid * ntiles + blockIdx.x] = s_h[tid];
}

// Exclusive scan of m values in three kernels: per-chunk sums, a scan of the
// chunk sums in one block, and the scan of each chunk from its offset.
constexpr int kScanChunk = kThreads * kItems;

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* s_warp, uint32_t* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) s_warp[w] = x;
  __syncthreads();
  if (w == 0) {
    uint32_t s = lane < kWarps ? s_warp[lane] : 0u;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, s, d);
      if (lane >= d) s += y;
    }
    if (lane < kWarps) s_warp[lane] = s;  // inclusive warp prefixes
  }
  __syncthreads();
  const uint32_t before = (w > 0 ? s_warp[w - 1] : 0u) + x - v;
  if (total) *total = s_warp[kWarps - 1];
  __syncthreads();
  return before;
}

__global__ void __launch_bounds__(kThreads) k_scan_sums(const uint32_t* in, long m, uint32_t* sums) {
  __shared__ uint32_t s_warp[kWarps];
  const long base = (long)blockIdx.x * kScanChunk;
  uint32_t acc = 0;
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    const long idx = base + (long)i * kThreads + threadIdx.x;
    if (idx < m) acc += in[idx];
  }
  uint32_t total;
  block_exclusive_scan(acc, s_warp, &total);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// One block: exclusive scan of the chunk sums, in place.
__global__ void __launch_bounds__(kThreads) k_scan_top(uint32_t* sums, int nchunks) {
  __shared__ uint32_t s_warp[kWarps];
  uint32_t carry = 0;
  for (int b0 = 0; b0 < nchunks; b0 += kThreads) {
    const int i = b0 + threadIdx.x;
    const uint32_t v = i < nchunks ? sums[i] : 0u;
    uint32_t total;
    const uint32_t ex = block_exclusive_scan(v, s_warp, &total);
    if (i < nchunks) sums[i] = carry + ex;
    carry += total;
  }
}

// Chunk element j lives at j + j / kItems in shared memory: a pad word after
// every kItems, so that both the coalesced pass (consecutive j per warp) and
// the per-thread pass (kItems consecutive j per thread) avoid bank conflicts.
__device__ __forceinline__ int padded(int j) { return j + j / kItems; }

__global__ void __launch_bounds__(kThreads) k_scan_apply(uint32_t* data, long m, const uint32_t* sums) {
  __shared__ uint32_t s_v[kScanChunk + kScanChunk / kItems];
  __shared__ uint32_t s_warp[kWarps];
  const long base = (long)blockIdx.x * kScanChunk;
  const int tid = threadIdx.x;
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    const long idx = base + (long)i * kThreads + tid;
    s_v[padded(i * kThreads + tid)] = idx < m ? data[idx] : 0u;
  }
  __syncthreads();
  uint32_t run[kItems], acc = 0;
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    run[i] = acc;
    acc += s_v[padded(tid * kItems + i)];
  }
  const uint32_t before = block_exclusive_scan(acc, s_warp, nullptr) + sums[blockIdx.x];
#pragma unroll
  for (int i = 0; i < kItems; ++i) s_v[padded(tid * kItems + i)] = before + run[i];
  __syncthreads();
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    const long idx = base + (long)i * kThreads + tid;
    if (idx < m) data[idx] = s_v[padded(i * kThreads + tid)];
  }
}

// Stable scatter of one tile.  Warp w owns the tile positions
// [w * 32 kItems, (w + 1) * 32 kItems); its lane l holds item i at position
// w * 32 kItems + 32 i + l, so (warp, item, lane) is position order.  Ranks
// among equal digits are counted per warp (lanes holding the same digit in
// one item round, plus the warp's running count of that digit), then offset
// by the counts of the lower warps; the tile is reordered by digit in shared
// memory and written out in runs of consecutive addresses.
template <bool FIRST, bool LAST>
__global__ void __launch_bounds__(kThreads) k_rs_scatter(const uint32_t* __restrict__ keys_in,
                                                         const uint32_t* __restrict__ vals_in,
                                                         const float* __restrict__ fmax, long n, int shift,
                                                         const uint32_t* __restrict__ offs, int ntiles,
                                                         uint32_t* keys_out, uint32_t* vals_out) {
  __shared__ uint32_t s_k[kTile];
  __shared__ uint32_t s_v[kTile];
  __shared__ uint32_t s_cnt[kWarps][kBins];  // per-warp digit counts, then per-warp digit offsets
  __shared__ uint32_t s_start[kBins], s_goff[kBins];
  __shared__ uint32_t s_warp[kWarps];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const long base = (long)blockIdx.x * kTile;
  const long seg = base + (long)w * 32 * kItems;
  const int valid = (int)((n - base) < kTile ? (n - base) : kTile);
  uint32_t key[kItems], val[kItems], rank[kItems];
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    const long idx = seg + 32 * i + lane;
    const bool in = idx < n;
    key[i] = in ? (FIRST ? fkey(__ldg(fmax + idx)) : __ldg(keys_in + idx)) : 0xffffffffu;
    val[i] = in ? (FIRST ? (uint32_t)idx : __ldg(vals_in + idx)) : 0u;
  }
  s_goff[tid] = offs[(size_t)tid * ntiles + blockIdx.x];
#pragma unroll
  for (int j = 0; j < kBins / 32; ++j) s_cnt[w][lane + 32 * j] = 0;
  __syncwarp();
  const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    const uint32_t d = (key[i] >> shift) & 255u;
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    const uint32_t before = s_cnt[w][d];
    __syncwarp();
    if ((peers & lt) == 0) s_cnt[w][d] = before + __popc(peers);
    __syncwarp();
    rank[i] = before + __popc(peers & lt);
  }
  __syncthreads();
  // digit tid: offsets of each warp's run within the digit, and the tile total
  uint32_t acc = 0;
#pragma unroll
  for (int j = 0; j < kWarps; ++j) {
    const uint32_t c = s_cnt[j][tid];
    s_cnt[j][tid] = acc;
    acc += c;
  }
  s_start[tid] = block_exclusive_scan(acc, s_warp, nullptr);
  __syncthreads();
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    const uint32_t d = (key[i] >> shift) & 255u;
    const uint32_t pos = s_start[d] + s_cnt[w][d] + rank[i];
    s_k[pos] = key[i];
    s_v[pos] = val[i];
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    const int pos = i * kThreads + tid;
    if (pos < valid) {
      const uint32_t k = s_k[pos];
      const uint32_t d = (k >> shift) & 255u;
      const size_t g = (size_t)s_goff[d] + (pos - s_start[d]);
      if (!LAST) keys_out[g] = k;
      vals_out[g] = s_v[pos];
    }
  }
}

// Number of the six periodic neighbours (+-1 along x, y, z) that come before
// particle q in the order: larger F_max, or equal F_max and smaller index.
// One block per (x, y) line; the six neighbour lines are read in step along z.
__global__ void __launch_bounds__(256) k_neighbours_before(const float* __restrict__ F, int nx, int ny, int nz,
                                                           uint8_t* out) {
  const int line = blockIdx.x;  // x ny + y
  const int x = line / ny, y = line - x * ny;
  const int xp = x + 1 == nx ? 0 : x + 1, xm = x == 0 ? nx - 1 : x - 1;
  const int yp = y + 1 == ny ? 0 : y + 1, ym = y == 0 ? ny - 1 : y - 1;
  const int lines[4] = {xp * ny + y, xm * ny + y, x * ny + yp, x * ny + ym};
  const int q0 = line * nz;  // nx ny nz < 2^31
  for (int z = threadIdx.x; z < nz; z += blockDim.x) {
    const int q = q0 + z;
    const float f = __ldg(F + q);
    const int zp = z + 1 == nz ? 0 : z + 1, zm = z == 0 ? nz - 1 : z - 1;
    int c = 0;
    const int zs[2] = {q0 + zp, q0 + zm};
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const float g = __ldg(F + zs[k]);
      c += (g > f) | ((g == f) & (zs[k] < q));
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int r = lines[k] * nz + z;
      const float g = __ldg(F + r);
      c += (g > f) | ((g == f) & (r < q));
    }
    out[q] = (uint8_t)c;
  }
}

}  // namespace

size_t fragment_scratch_bytes(long n3) {
  const long ntiles = (n3 + kTile - 1) / kTile;
  const long m = ntiles * kBins;
  const long nchunks = (m + kScanChunk - 1) / kScanChunk;
  return (size_t)n3 * 16 + (size_t)m * 4 + (size_t)nchunks * 4 + 256;
}

cudaError_t fragment_order(const float* fmax, int nx, int ny, int nz, void* scratch, int32_t* order,
                           uint8_t* n_before, cudaStream_t st) {
  const long n3 = (long)nx * ny * nz;
  if (n_before) {
    k_neighbours_before<<<(unsigned)(nx * ny), nz < 256 ? ((nz + 31) / 32) * 32 : 256, 0, st>>>(fmax, nx, ny, nz,
                                                                                              n_before);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (!order) return cudaSuccess;
  const int ntiles = (int)((n3 + kTile - 1) / kTile);
  const long m = (long)ntiles * kBins;
  const int nchunks = (int)((m + kScanChunk - 1) / kScanChunk);
  uint32_t* ka = static_cast<uint32_t*>(scratch);
  uint32_t* va = ka + n3;
  uint32_t* kb = va + n3;
  uint32_t* vb = kb + n3;
  uint32_t* hist = vb + n3;
  uint32_t* sums = hist + m;
  const uint32_t *kin = nullptr, *vin = nullptr;
  for (int pass = 0; pass < 4; ++pass) {
    const int shift = 8 * pass;
    uint32_t* kout = (pass & 1) ? kb : ka;
    uint32_t* vout = pass == 3 ? reinterpret_cast<uint32_t*>(order) : ((pass & 1) ? vb : va);
    if (pass == 0) k_rs_hist<true><<<ntiles, kThreads, 0, st>>>(nullptr, fmax, n3, shift, hist, ntiles);
    else k_rs_hist<false><<<ntiles, kThreads, 0, st>>>(kin, nullptr, n3, shift, hist, ntiles);
    k_scan_sums<<<nchunks, kThreads, 0, st>>>(hist, m, sums);
    k_scan_top<<<1, kThreads, 0, st>>>(sums, nchunks);
    k_scan_apply<<<nchunks, kThreads, 0, st>>>(hist, m, sums);
    if (pass == 0)
      k_rs_scatter<true, false><<<ntiles, kThreads, 0, st>>>(nullptr, nullptr, fmax, n3, shift, hist, ntiles, kout, vout);
    else if (pass < 3)
      k_rs_scatter<false, false><<<ntiles, kThreads, 0, st>>>(kin, vin, nullptr, n3, shift, hist, ntiles, kout, vout);
    else
      k_rs_scatter<false, true><<<ntiles, kThreads, 0, st>>>(kin, vin, nullptr, n3, shift, hist, ntiles, nullptr, vout);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    kin = kout;
    vin = vout;
  }
  return cudaSuccess;
}

int fragment_kernels(bool order, bool counts) { return (order ? 4 * 5 : 0) + (counts ? 1 : 0); }

}  // namespace pin
