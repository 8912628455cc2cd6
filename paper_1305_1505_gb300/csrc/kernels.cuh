// Launch interface of the collapse-time passes (kernels.cu).
//
// Spectral arrays are half-spectra stored [kx][ky][kz] with kz padded to an
// even stride NHP >= N/2+1 (pad modes are zero), complex64.  The filtered
// Hessian spectrum of Sec. 2.1.1,
//   T_ij(k) = (k_i k_j / k^2) W(kR) delta(k),
// is separable once Phi0 = delta / k^2 is formed (once per field):
//   T_ij = mx(kx) my(ky) mz(kz) Phi0,   m in {W, k W, k^2 W} per axis
// (W = exp(-k^2 R^2/2) = Wx Wy Wz, and k carries a zero on the Nyquist index
// for the odd multipliers), so the x pass needs three transforms and only the
// y and z passes carry all six components.
#pragma once
#include <cuda.h>  // CUtensorMap (the encoder itself is fetched from the driver at run time)
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace pin {

constexpr int kMaxFields = 9;

// x pass (lines of length nx): for each output f, dst[f] = IDFT_x(mult[xm[f]]
// * src).  The source tiles arrive by TMA: tm is a 2D map over src,
// {ny*nhp columns, batch*nx rows} (realisations stacked along rows), box
// {tc, nx/boxes}.
struct ArgsX {
  CUtensorMap tm;
  const float2* src;
  float2* dst[3];
  int xm[3];
  int nout;
  int ny;             // rows of a plane: the columns are (ky, kz), ny * nhp of them
  const float* mult;  // [3][nx] multipliers of this radius (W, kW, k^2W, each / nx)
  const float2* tw;   // twiddles: w_N^{p k1} [E][P], then w_P^{p1 k2a} [P2][P1] for three levels
  int nhp;
  int batch;          // realisations stacked back to back (same N, radii)
  int* err;           // set to 1 if a TMA wait gave up (bounded wait)
  long long wait_cycles;  // budget of a TMA wait in SM clocks; <= 0: the default (2^31)
  CUtensorMap tm_out[3];  // maps of dst[f] (filled at launch when outputs go out by TMA stores)
};

// y pass (lines of length ny): dst[f] = zfac[f](kz) * IDFT_y(mult[ym[f]] *
// src[sel[f]]), where the z factor mult_z[zm[f]](kz), times i when muli[f], is
// constant along a y line.  Outputs are processed in the given order;
// consecutive outputs with the same source share one staged tile.  tm is a 4D
// map over the three source spectra (stored back to back),
// {nhp, ny, batch*nx, 3}, box {tc, ny/boxes, 1, 1}.
struct ArgsY {
  CUtensorMap tm;
  const float2* src[3];
  float2* dst[kMaxFields];
  int sel[kMaxFields];
  int ym[kMaxFields];
  int zm[kMaxFields];
  int muli[kMaxFields];
  // optional second store of the same transform with its own z factor
  float2* dst2[kMaxFields];
  int zm2[kMaxFields];
  int muli2[kMaxFields];
  int nout;
  int nx, nz;           // x planes per realisation; z line length (z factors for kz <= nz/2)
  const float* mult;    // [3][ny] y multipliers
  const float* mult_z;  // [3][nz] z multipliers
  const float2* tw;
  int nhp;
  int batch;
  int* err;
  long long wait_cycles;
  CUtensorMap tm_out[kMaxFields];  // maps of dst[o] (filled at launch when outputs go out by TMA stores)
};

// A particle whose FP32 collapse is ill-conditioned, finished in FP64 by the
// redo kernel: kind 0 (near-degenerate eigenvalue pair, queued by the z pass)
// carries the six FP32 Hessian components; kind 1 (near-tangent or
// unconverged root, queued by the root kernel) carries the three eigenvalues
// in h[0..2].
struct RedoEntry {
  int q;
  float h[6];
  int kind;
};

// z pass: c2r of each field (its z factor already applied by the y pass),
// then either the eigenvalues of every particle (lam_out, [3][nlines*N];
// NaN for particles queued for the FP64 redo), or, where z_fuses_roots, the
// collapse times and running maximum directly, or a dump of the real fields.
struct ArgsZ {
  const float2* src[kMaxFields];
  int nfields;
  int nlines;    // batch * N^2 lines along z
  int npart;     // batch * N^3 particles
  int prefetch_blocks;  // z pass: prefetch the lines of block + this many into L2 (0: none)
  const float2* tw;
  int nhp;
  // eigenvalue mode (nfields 6), plus the displacement components (nfields 9)
  float* lam_out;
  float* psi_out;   // [3][npart] smoothed displacement of this radius
  float* vstate;    // [3][npart] displacement at R_max, or null
  // root and redo kernels
  float* fmax;
  int* idx;
  int scale;
  int correction;
  float dcorr_f;
  double dcorr_d;
  float tau_eig;   // FP64 redo when |r| > 1 - tau_eig
  float tau_root;  // FP64 redo when kappa < tau_root
  unsigned long long* counters;  // [0] eigen redo, [1] root redo, [2] list overflow
  RedoEntry* redo_list;          // FP64 redo queue of this radius
  unsigned* redo_count;          // zeroed before the z pass
  unsigned redo_cap;
  // dump mode
  float* out[kMaxFields];
};

struct PassShape {
  int E, P;
  int P1, P2;     // P = P1 * P2; P2 > 1: three-level line transform
  int tc;         // columns per block, x/y passes
  int lines;      // lines per block, z pass
  size_t smem_xy; // dynamic shared bytes, x/y passes
  size_t smem_z;
  int threads_xy, threads_z;
};

// Tensor maps of the x and y passes (host; the encoder comes from the driver
// entry point, so no driver library is linked).  spec_elems is the stride
// between the spectra the y map spans; tc is the tile width (columns) of the
// pass that reads the map, one of xy_tile_options.
cudaError_t make_tmap_x(CUtensorMap* tm, const float2* src, int nx, int ny, int nhp, int batch, int tc);
// 2D map of rows of `cols` complex values (row pitch cols), box {tc, box_rows}
cudaError_t make_tmap_rows(CUtensorMap* tm, const float2* base, int cols, long long rows, int tc, int box_rows);
cudaError_t make_tmap_y(CUtensorMap* tm, const float2* src3, int nx, int ny, int nhp, size_t spec_elems,
                        int batch, int tc);
// Radix schedules of the x/y line transforms (fft.cuh ShapeBase<N, V>):
// 0, the default and the z pass's, and 1.
constexpr int kRadixVariants = 2;
// Tile widths the x/y pass over lines of n points can run with radix
// schedule v (opts[0] is the default); returns their number (0 for an
// unsupported size or schedule).
int xy_tile_options(int n, int v, int* opts);

bool size_supported(int n);
PassShape pass_shape(int n);          // schedule 0: z pass, and the x/y defaults
PassShape pass_shape_xy(int n, int v);  // the x/y line transform of schedule v
cudaError_t prepare_kernels(int n);  // sets shared-memory attributes (once per device)
// tc: tile width, one of xy_tile_options(n, v) (anything else runs the
// default of schedule v); v: radix schedule
cudaError_t launch_x(int n, int tc, int v, const ArgsX& a, cudaStream_t st);
cudaError_t launch_y(int n, int tc, int v, const ArgsY& a, cudaStream_t st);
// schedule 1 (kernels_v1.cu)
cudaError_t upload_constant_twiddles_v1();  // that unit's copy of the register-DFT twiddles
cudaError_t prepare_xy_v1(int n);
int xy_tile_options_v1(int n, int* opts);
PassShape pass_shape_xy_v1(int n);
cudaError_t launch_x_v1(int n, int tc, const ArgsX& a, cudaStream_t st);
cudaError_t launch_y_v1(int n, int tc, const ArgsY& a, cudaStream_t st);
cudaError_t launch_z(int n, const ArgsZ& a, bool dump, cudaStream_t st);
// Second-order LPT pieces: the z pass writing the source S of every particle
// (from the six fields in src[0..5]) to out[0]; the inverse-sign transform
// along z of real lines (nlines of them, an even number) into a padded
// half-spectrum; and Phi2 = scale conj(T) / k^2.
cudaError_t launch_z_source(int n, const ArgsZ& a, cudaStream_t st);
cudaError_t launch_fwd_z(int n, const float* src, float2* dst, int nlines, int nhp, const float2* tw,
                         cudaStream_t st);
cudaError_t launch_phi2(const float2* T, float2* out, int nx, int ny, int nz, int nhp, double box, float scale,
                        cudaStream_t st);
// True when the z pass of size n also computes the collapse times and the
// running maximum (launch_roots is then not called for that size).
bool z_fuses_roots(int n);
// Collapse time and running maximum from the eigenvalues the z pass wrote
// (after it, same stream), then the FP64 redo of every queued particle.
cudaError_t launch_roots(const ArgsZ& a, cudaStream_t st);
cudaError_t launch_redo(const ArgsZ& a, cudaStream_t st);
cudaError_t upload_constant_twiddles();  // per device

// Host helpers shared by the plan path (pin.cu) and the allocation-free entry
// point (noalloc.cu), so that both build identical tables:
//   padded_half      kz stride of the padded half-spectra (n/2 + 1 rounded up
//                    to a multiple of 4 complex values)
//   correction_dcorr 1/delta_c - 1/x3 of the quasi-spherical correction
//   fill_mult        {W, kW, k^2 W} / n of one axis at one radius ([3][n])
//   fill_twiddles    the line transform's twiddles of one axis
//   launch_load_phi0 Phi0 = delta / k^2 into the padded layout (C64 or C128
//                    input, batch realisations back to back)
int padded_half(int n);
double correction_dcorr();
void fill_mult(float* out, int n, double box, double radius);
void fill_twiddles(float2* t, int n, const PassShape& sh);
cudaError_t launch_load_phi0(const void* src, int dtype, int nx, int ny, int nz, int nhp, double box, int batch,
                             float2* phi0, cudaStream_t st);

// All-FP64 loop of a PIN_FP64 plan (fp64.cu): device bytes of its workspace
// (FP64 half-spectrum, one full complex cube, the tensor, F_max), the input
// as an FP64 half-spectrum, the whole radius loop into fmax / idx (N^3 each,
// strict running maximum from 0 / -1), and the FP32 copy of F_max.
size_t fp64_workspace_bytes(int nx, int ny, int nz);
cudaError_t fp64_load(const void* src, int dtype, int nx, int ny, int nz, double2* d64, cudaStream_t st);
cudaError_t fp64_collapse(const double2* d64, int nx, int ny, int nz, double box, int nscales, const double* radii,
                          int correction, double dcorr, double2* work, double* h6, double* fmax, int* idx,
                          cudaStream_t st);
cudaError_t fp64_cast(const double* in, size_t n3, float* out, cudaStream_t st);

// Seeded initial conditions on the device (ic_gpu.cu): batch cubic
// half-spectra [n][n][n/2+1] complex64 into out, realisation b keyed by
// keys_dev[b] (the splitmix64 of its seed), amplitude amp of P(k).
cudaError_t generate_ic(int n, double box, const uint64_t* keys_dev, int batch, double amp, double ns,
                        double gamma, float2* out, cudaStream_t st);

// Fragmentation front end (fragment.cu): the particles of one nx*ny*nz grid in
// descending F_max (ties: ascending index) into `order`, and the number of
// their six periodic neighbours that precede them into `n_before`; either
// output may be null.  `scratch` holds fragment_scratch_bytes(N^3) bytes.
size_t fragment_scratch_bytes(long n3);
cudaError_t fragment_order(const float* fmax, int nx, int ny, int nz, void* scratch, int32_t* order,
                           uint8_t* n_before, cudaStream_t st);
int fragment_kernels(bool order, bool counts);  // launches of one fragment_order call

}  // namespace pin
