/*
 * pin.h -- C-ABI of libpin.so, the GB300 (sm_103a) collapse-time path of the
 * PINOCCHIO method (Monaco et al. 2013, Sec. 2.1.1 "Collapse times").
 *
 * The problem, as the paper states it: a Gaussian linear density field
 * delta_l on an N^3 grid of side L (Sec. 2.1.1, Eq. "deltal") is filtered with
 * a Gaussian window at each of several radii R; for each R inverse FFTs give the
 * deformation tensor (Hessian of the peculiar potential), and per grid point
 * ("particle") the ellipsoidal truncation of third-order LPT with its
 * quasi-spherical correction gives the inverse collapse time F = 1/D(t_coll)
 * (Eq. F).  Each particle keeps the highest F along its trajectory, F_max, and
 * the radius R_max at which it was reached.
 *
 * Conventions shared by every call:
 *  - Every call returns a pin_status; nothing throws across the ABI.  The text
 *    of the last error of a plan is available from pin_last_error().
 *  - The caller owns every input and output buffer; the plan owns all device
 *    workspace (pin_footprint_bytes() tells how much).
 *  - Half-spectra are [nx][ny][nz/2+1] complex, row major, index
 *    (ix*ny + iy)*(nz/2+1) + iz; the signed wavenumber index of i along an
 *    axis of n points is i for i < n/2 and i - n otherwise (the Nyquist index
 *    is -n/2), k = 2 pi s / L with L the side of that axis in Mpc/h.  DFT
 *    convention: d(q) = (nx ny nz)^-1 sum_k D(k) e^{+i k.q}; the kz = 0 and
 *    kz = nz/2 planes must be Hermitian (D(-kx,-ky) = conj D(kx,ky)).
 *    "N^3" below stands for nx*ny*nz.
 *  - Real fields are [nx][ny][nz] row major, q = (x*ny + y)*nz + z.
 *  - Calls on one plan are not re-entrant; different plans may be used from
 *    different threads.  Work is enqueued on the plan's CUDA stream.
 *  - No call makes a device wait without bound: pin_sync() takes a timeout.
 */
#ifndef PIN_H
#define PIN_H

#include <stddef.h>
#include <stdint.h>

#include "pin_ic.h" /* pin_spectrum */

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pin_plan_s* pin_plan_t;

typedef enum {
  PIN_OK = 0,
  PIN_EINVAL = 1,   /* bad argument: size, radius, pointer, dtype, scale index */
  PIN_ENOMEM = 2,   /* device allocation failed (nothing is left allocated) */
  PIN_ECUDA = 3,    /* a CUDA runtime call failed; see pin_last_error() */
  PIN_EBUSY = 4,    /* reserved for admission control above this library */
  PIN_ETIMEOUT = 5, /* pin_sync() expired before the plan's work finished */
  PIN_ESTATE = 6    /* call out of order, e.g. collapse times before pin_set_ic */
} pin_status;

enum { PIN_CORR_NONE = 0, PIN_CORR_SPHERE = 1 };
enum { PIN_FP32_FALLBACK64 = 0, PIN_FP64 = 1 };
enum { PIN_C64 = 0, PIN_C128 = 1 };

typedef struct {
  int nx, ny, nz;        /* grid, each in {8,16,32,48,64,96,128,192,256,384,512,768}; they
                            may differ (non-cubic boxes are allowed by the paper's code,
                            Sec. 2.1.1); the cells are cubic */
  double box;            /* side along x in Mpc/h, > 0; the sides along y and z are
                            box ny / nx and box nz / nx */
  int nscales;           /* number of radii S, 1..64 */
  const double* radii;   /* S radii in Mpc/h (Gaussian sigma, >= 0); copied at pin_plan;
                            processed in the given order, index 0 first (callers
                            normally give the largest radius first, as the
                            trajectories of Sec. 2.1.1 run from large to small R) */
  int correction;        /* PIN_CORR_SPHERE (quasi-spherical correction, default) or
                            PIN_CORR_NONE (pure ellipsoidal 3LPT truncation) */
  int precision;         /* PIN_FP32_FALLBACK64: FP32 FFTs and collapse, FP64 redo of
                            near-degenerate eigenvalues and near-tangent roots.
                            PIN_FP64: a slow all-FP64 loop for checking (filter, line
                            transforms, eigenvalues, collapse and running maximum in
                            double; pin_collapse_times_f64 returns F_max in FP64); batch 1,
                            no velocities; only the collapse-time calls use it, the
                            other calls of the plan run in FP32 */
  void* stream;          /* cudaStream_t to run on, or NULL for a plan-owned stream */
  int batch;             /* number of realisations B processed together (0 or 1: one);
                            they share N, box, radii and correction.  Inputs and outputs
                            are then B consecutive copies of the single-realisation
                            layout; one launch per pass covers all of them.  B * N^3 must
                            stay below 2^31.  pin_hessian and pin_displacements need B = 1. */
  int velocities;        /* 1: also keep, per particle, the Zel'dovich displacement of the
                            field smoothed at R_max (the velocity of Sec. 2.1.1, see
                            pin_velocities); costs three more spectra per radius.  0: off. */
} pin_plan_desc;

/* Runtime counters of a plan (cumulative over its pin_collapse_times calls). */
typedef struct {
  uint64_t eig_fp64_redo;   /* particle-scales redone in FP64 for a near-degenerate pair */
  uint64_t root_fp64_redo;  /* particle-scales redone in FP64 for a near-tangent root */
  uint64_t fp64_queue_overflow; /* of those, kept at FP32 because the redo queue of a
                                   radius (1/64 of the grid) was full */
  uint64_t collapse_calls;  /* completed pin_collapse_times calls */
} pin_stats;

/* Creates a plan: validates the description, allocates the device workspace
 * on the current CUDA device, and builds the per-radius filter tables.
 * On error *out is NULL and nothing stays allocated. */
pin_status pin_plan(pin_plan_t* out, const pin_plan_desc* d);

/* Device bytes a plan with this description would allocate (0 if invalid). */
size_t pin_footprint_bytes(const pin_plan_desc* d);

/* Loads the linear density field delta(k) (Sec. 2.1.1, Eq. "deltal"), a
 * half-spectrum as described above (B of them back to back for a batch), dtype PIN_C64 (interleaved float) or
 * PIN_C128 (interleaved double, rounded to FP32 on the device), from host
 * memory (on_device = 0) or device memory (on_device = 1).  Page-locked host
 * input is read in place by the device (no staging copy); other host memory
 * is copied in first.  The data are copied; the caller may reuse its buffer
 * when the call returns (host input) or once the plan's stream has passed
 * this point (device input). */
pin_status pin_set_ic(pin_plan_t p, const void* delta_k, int dtype, int on_device);

/* Generates delta(k) on the device from a seed instead of loading it: the
 * seeded Gaussian field of include/pin_ic.h (P(k) = A k^ns T_BBKS(k/Gamma)^2
 * normalised to sigma8, splitmix64 keyed on (seed, linear mode index),
 * Box-Muller), computed per mode in FP64 and rounded to FP32; realisation b of
 * a batch uses seed + b.  The paper generates its linear field with N-GenIC
 * (Sec. 2.2); this generator stands in for it.  Equal to pin_set_ic of the
 * host module's FP32 field up to the last bits of the device's FP64 math
 * functions (they may differ from the host's by an ulp, which survives the
 * rounding to FP32 for about one mode in 1e8).  Cubic grids only. */
pin_status pin_set_ic_seed(pin_plan_t p, uint64_t seed, const pin_spectrum* ps);

/* Runs the whole collapse-time loop over all radii (Sec. 2.1.1): filter,
 * inverse 3D FFTs of the six Hessian components, eigenvalues, collapse time F,
 * running maximum.  Outputs (caller-owned, N^3 each, real-field layout):
 *   F_max[q]     highest F over all radii, 0 if the particle never collapses;
 *   scale_idx[q] index of the radius where F_max was reached (first such
 *                index on exact ties), -1 if never collapses.
 * on_device = 1: both are device pointers; the call only enqueues work and
 * returns (use pin_sync or the stream).  on_device = 0: host pointers; the
 * call returns when the results are in host memory (page-locked host memory
 * is written by the device through its mapping, other host memory by a copy). */
pin_status pin_collapse_times(pin_plan_t p, float* F_max, int32_t* scale_idx, int on_device);

/* pin_collapse_times of a PIN_FP64 plan with F_max in double precision
 * (F_max: N^3 doubles; scale_idx as in pin_collapse_times).  PIN_EINVAL for a
 * plan of another precision. */
pin_status pin_collapse_times_f64(pin_plan_t p, double* F_max, int32_t* scale_idx, int on_device);

/* v_max of Sec. 2.1.1: for each particle, the gradient of the potential
 * (smoothed on R_max), taken as the linear (Zel'dovich) displacement
 * psi_R(k) = i k W(kR) delta(k)/k^2 at the radius where F_max was reached
 * (zero where the particle never collapses), from the last
 * pin_collapse_times call of a plan created with velocities = 1.  Output
 * psi_max = [3][B][N^3] floats in Mpc/h; the peculiar velocity follows by the
 * linear factor a H f(a) of the caller's cosmology (D = 1 at z = 0).  Same
 * on_device semantics as pin_collapse_times. */
pin_status pin_velocities(pin_plan_t p, float* psi_max, int on_device);

/* Second-order LPT displacement of the unsmoothed field, for halo positions
 * beyond the Zel'dovich approximation (Sec. 4 names 2LPT as the next step for
 * them; the formula is the standard one of second-order Lagrangian
 * perturbation theory).  With phi_ij the deformation tensor at R = 0 (the
 * Hessian of pin_hessian, unsmoothed) and its second invariant
 *   S(q) = sum_{i<j} (phi_ii phi_jj - phi_ij^2),
 *   psi2(k) = (3/7) i k S(k) / k^2,
 * so that div psi2 = -(3/7) S and, with D2 = -(3/7) D^2, the position is
 * x = q + D psi + D^2 psi2 (psi from pin_displacements).  Output
 * psi2 = [3][N^3] floats in Mpc/h (odd-order Nyquist modes zeroed as for
 * psi).  Uses the plan's spectra as scratch (batch 1 only; any collapse state
 * is kept, the next pin_collapse_times rebuilds the spectra).  Same on_device
 * semantics as pin_collapse_times. */
pin_status pin_displacements_2lpt(pin_plan_t p, float* psi2, int on_device);

/* Fragmentation front end (Sec. 2.1.2): the fragmentation considers the
 * particles in descending F_max (an effectively chronological order) and,
 * for each, the halos its six neighbours belong to.  From the F_max of the
 * plan's last pin_collapse_times call (batch 1 only):
 *   order[i]     (N^3 int32) the particle index q of the i-th particle in
 *                descending F_max; equal F_max in ascending q (a reading: the
 *                paper gives no tie rule), so order is a permutation of [0, N^3);
 *   n_before[q]  (N^3 uint8) how many of the six periodic neighbours of q
 *                (q +- 1 along x, y and z) come before q in that order; 0 marks
 *                a peak of the F_max field (a new halo, case (i)).
 * Either output may be NULL (skipped), not both.  Runs on the plan's stream
 * and uses the y-pass spectra as scratch (they are rebuilt by the next
 * pin_collapse_times).  Same on_device semantics as pin_collapse_times.
 * PIN_ESTATE before the first pin_collapse_times, PIN_EINVAL for batch > 1. */
pin_status pin_fragment_order(pin_plan_t p, int32_t* order, uint8_t* n_before, int on_device);

/* The six real components of the deformation tensor phi_ij(q) at radius
 * index `scale` (the a1-a2 steps alone), out6 = [6][N^3] floats in the order
 * xx, yy, zz, xy, xz, yz.  Same on_device semantics as pin_collapse_times. */
pin_status pin_hessian(pin_plan_t p, int scale, float* out6, int on_device);

/* Zel'dovich (first-order LPT) displacement of the unsmoothed field,
 * psi(k) = i k delta(k) / k^2 (so that delta = -div psi), Sec. 2.1.2:
 * out psi = [3][N^3] floats (x, y, z components, Mpc/h).  Odd-order Nyquist
 * modes are zeroed.  Same on_device semantics as pin_collapse_times. */
pin_status pin_displacements(pin_plan_t p, float* psi, int on_device);

/* Waits for the plan's enqueued work, polling; PIN_ETIMEOUT after timeout_ns
 * nanoseconds (timeout_ns < 0: no limit).  The device is never made to wait. */
pin_status pin_sync(pin_plan_t p, int64_t timeout_ns);

pin_status pin_get_stats(pin_plan_t p, pin_stats* out);

/* Number of kernels one pin_collapse_times call launches (for accounting):
 * per radius the x, y and z passes, the root pass unless the z pass of this
 * grid size computes the collapse times itself (N = 384 and 768, the sizes
 * with three-level line transforms), and the FP64 redo. */
int pin_kernels_per_call(pin_plan_t p);

/* Measurement hooks.  pin_profile(p, 1) makes later pin_collapse_times calls
 * record CUDA events around each pass of each radius (on the plan's stream,
 * inside its graph); pin_pass_times() then waits for the plan's work and
 * returns, for the last completed call, the device time in milliseconds summed
 * over radii of: ms4[0] the x pass (filter + transform), ms4[1] the y pass,
 * ms4[2] the z pass (c2r + eigenvalues; at N = 384 and 768 also the collapse
 * time and running max), ms4[3] the root pass (collapse time + running max, where it
 * is a kernel of its own) with the FP64 redo of the queued ill-conditioned
 * particles.  Each is measured on the stream its pass runs on; under an
 * overlapped schedule (pin_set_schedule) the passes overlap, so the four sums
 * exceed the call's time. */
pin_status pin_profile(pin_plan_t p, int enable);
pin_status pin_pass_times(pin_plan_t p, double* ms4);

/* Tile and radix schedules of the x and y passes (the paper has no
 * counterpart: its FFTs are FFTW's).  Each of those passes transforms blocks
 * of tc columns of the spectrum at a time, every line by a decomposition of
 * its length n = E x P (E values per thread, P threads per line; P = P1 x P2,
 * a second shared-memory exchange when P2 > 1).  Each length has
 * pin_radix_schedules() such decompositions ("radix schedules"); schedule 0
 * is the default and the z pass's.  Every tile width computes each column's
 * line transform with the same arithmetic, so the tile width changes timings,
 * never results; the radix schedule changes the order of the arithmetic, so
 * results differ in the last bits (both are checked against the oracle).
 *
 * pin_tile_options: the widths a pass over lines of n points can run with
 * radix schedule 0, the default first, into opts[0 .. *count - 1]
 * (*count <= 2); pin_tile_options_radix: the same for schedule `radix`.
 * PIN_EINVAL for an unsupported n or schedule.
 * pin_radix_shape: E, P1, P2 of schedule `radix` for lines of n points.
 * pin_get_tiles / pin_set_tiles: the widths the plan runs for its x pass
 * (lines of nx points) and y pass (ny points); 0 selects the default of the
 * plan's radix schedule, any other value must be one of its options (else
 * PIN_EINVAL, plan unchanged).  Setting waits for the plan's stream.
 * pin_get_radix / pin_set_radix: the radix schedules of the plan's x and y
 * passes (set: waits for the plan's stream, keeps the tile widths where the
 * new schedules run them, else their defaults).
 * pin_autotune: times every (radix schedule, tile width) candidate of the x
 * pass and of the y pass on the plan's own buffers (reps launches each,
 * 1..1000, after one untimed launch; the first radius, the plan's mode) and
 * keeps the fastest of each.  Only the plan's workspaces are written (Phi0 is
 * zeroed first if no field is set); F_max, the scale index and v_max are
 * untouched.  Choices are kept per (device, nx, ny, nz, batch, velocities)
 * for the process: a later call for the same shape applies the kept choice
 * without timing unless flags has PIN_TUNE_FORCE.  The chosen widths go to
 * *tc_x and *tc_y (either may be NULL; pin_get_radix gives the schedules).
 * PIN_ESTATE while the plan's stream is being captured. */
#define PIN_TUNE_FORCE 1
pin_status pin_tile_options(int n, int* opts, int* count);
pin_status pin_tile_options_radix(int n, int radix, int* opts, int* count);
int pin_radix_schedules(void);
pin_status pin_radix_shape(int n, int radix, int* E, int* P1, int* P2);
pin_status pin_get_tiles(pin_plan_t p, int* tc_x, int* tc_y);
pin_status pin_set_tiles(pin_plan_t p, int tc_x, int tc_y);
pin_status pin_get_radix(pin_plan_t p, int* vx, int* vy);
pin_status pin_set_radix(pin_plan_t p, int vx, int vy);
pin_status pin_autotune(pin_plan_t p, int reps, int flags, int* tc_x, int* tc_y);

/* Replaces the plan's radius list (1..64 radii, as in pin_plan_desc) without
 * touching its device workspace, so that one plan serves requests with other
 * radii: a server keeps plans per grid size and reuses them.  Waits for the
 * plan's stream, then uploads the new filter tables.  The graph captured for
 * a radius count is kept, so returning to a count seen before needs no new
 * capture.  The next pin_collapse_times uses the new radii; pin_hessian's scale
 * index refers to them.  PIN_EINVAL for a bad list (plan unchanged). */
pin_status pin_set_radii(pin_plan_t p, int nscales, const double* radii);

/* Radius schedule of pin_collapse_times (the paper has no counterpart; its
 * loop is sequential).  0 (default): the passes of each radius run in order on
 * the plan's stream.  1: the z pass and FP64 redo of radius s run on a second,
 * lower-priority stream while the x pass of radius s + 1 runs; the y pass of
 * s + 1 waits for them.  2: the x and y passes of radius s + 1 both overlap the
 * z pass of radius s, the y pass writing a second set of spectra (six more, nine
 * with velocities: pin_footprint_bytes does not count them), and the y pass of
 * s + 2 waits for the z pass of s.  Results are bit-identical in every
 * schedule; only the time changes (the z pass is bound by instruction issue,
 * the x/y passes by memory).  Needs a grid whose z pass computes the collapse
 * times itself (nz = 384 or 768), else PIN_EINVAL.  Waits for the plan's
 * stream; the next call re-captures its graph.  PIN_ENOMEM (plan unchanged)
 * when the second set of spectra does not fit. */
pin_status pin_set_schedule(pin_plan_t p, int schedule);
int pin_get_schedule(pin_plan_t p);

/* Failure paths, exercised without any GPU fault (the paper has no
 * counterpart; its code is an MPI job).
 *
 * pin_set_wait_budget: the budget, in SM clock cycles, of each bounded wait of
 * the x and y passes for a staged transfer (0: the default, 2^31 cycles, about
 * a second).  A block whose wait runs out waits once more, with the default
 * budget, for its transfers in flight, sets the plan's error word and returns;
 * the next pin_sync (or host-output call) reports PIN_ECUDA once ("results are
 * invalid") and clears the word, so the plan stays usable.  A tiny budget
 * makes the waits run out on purpose.  Waits for the plan's stream; PIN_EINVAL
 * for a negative budget.
 *
 * pin_debug_fail_alloc: host-side allocation-failure injection.  With
 * nth >= 0, the device allocation with index nth (counted from 0 over the
 * allocations of later pin_plan calls of the process) fails as if the device
 * were out of memory; pin_plan then returns PIN_ENOMEM and frees what it had
 * allocated.  The injection is used up by that failure; nth < 0 cancels it. */
pin_status pin_set_wait_budget(pin_plan_t p, int64_t cycles);
void pin_debug_fail_alloc(int nth);

/* Largest grid side the no-allocation entry point below accepts. */
#define PIN_NOALLOC_MAX_N 64

/* pin_collapse_times without any device allocation, for callers that cannot
 * allocate at call time: a serving process whose pool already holds all the
 * memory it may use, code running inside an allocator hook, or a latency-
 * critical caller that cannot accept cudaFree's implicit device-wide
 * synchronisation.  (The paper has no counterpart; this is an interface
 * convenience over the same passes.)
 *
 * Inputs and outputs are device pointers owned by the caller: delta_k is the
 * half-spectrum (dtype PIN_C64 or PIN_C128, layout as for pin_set_ic), radii
 * the nscales radii in host memory, F_max and scale_idx the N^3 outputs, with
 * the meaning of pin_collapse_times and the same values bit for bit (the same
 * tables, kernels and FP64 redo capacity run).  Work is enqueued on `stream`
 * (NULL: the legacy default stream) and the call returns without waiting for
 * the kernels; the per-radius tables are copied in from a static host staging
 * area on that stream, a copy from pageable memory that may wait for the
 * stream's earlier work.
 *
 * The workspace is one static device array of 13.9 MB, sized for
 * n <= PIN_NOALLOC_MAX_N, which every GPU that loads this library holds until
 * the process exits.  Larger n returns PIN_EINVAL, as do the argument errors
 * of pin_plan.  The first call on a device sets that device up (looks up the
 * array's address, loads constant tables, sets kernel limits); make it before
 * any stream capture.  All calls share the array and it keeps the previous
 * call's contents (each call rewrites everything it reads and clears its
 * counters and error word); calls whose work overlaps on the GPU race on it,
 * so the caller must serialise them. */
pin_status pin_collapse_times_noalloc(const void* delta_k, int dtype, int n, double box,
                                      int nscales, const double* radii, int correction,
                                      float* F_max, int32_t* scale_idx, void* stream);

/* What the last pin_collapse_times_noalloc call on the current device
 * recorded, read from the shared workspace without allocating; call it only
 * after that call's stream has completed (otherwise the values are those of
 * work still in flight).  *wait_failed = 1 when a transfer wait of the x or y
 * pass gave up (its bounded wait ran out; the outputs are then invalid and the
 * call returns PIN_ECUDA).  counters3[0] and [1]: particle-scales redone in
 * FP64 for a near-degenerate eigenvalue pair and for a near-tangent root;
 * counters3[2]: of those, kept at FP32 because the redo queue of a radius was
 * full (as in pin_stats).  PIN_ESTATE if no call has run on this device. */
pin_status pin_noalloc_status(int* wait_failed, uint64_t* counters3);

const char* pin_strerror(pin_status s);
const char* pin_last_error(pin_plan_t p);

/* Releases the plan and its device workspace (waits for its work first). */
void pin_destroy(pin_plan_t p);

#ifdef __cplusplus
}
#endif
#endif
