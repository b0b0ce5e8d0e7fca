/*
 * pxc: line-list -> line intensities -> cross sections on one B300 (sm_103a).
 *
 * C ABI of the hot path of PyExoCross 2.0 (Zhang, Yurchenko, Tennyson):
 * partition functions (Sec. 2.4.2, Eq. pf; Sec. 3.1, Eq. Q nlte 2T), LTE and
 * two-temperature absorption intensities (Sec. 3.2, Eqs. abs intensity lte,
 * nlte v, nlte ab 2T), and cross sections on a wavenumber grid with a line-wing
 * cut-off (Sec. 2.4.3, Eq. xsec; Table profile: Doppler/Gaussian, Lorentzian,
 * Voigt), plus the adjoint of a linear functional of the cross section.
 *
 * Conventions shared by every call
 *  - Every array argument is a DEVICE pointer owned by the caller, unless the
 *    name says "host".  The library never frees caller memory.
 *  - The library allocates no device memory after pxc_workspace_create: all
 *    scratch lives in the caller-provided buffer given to pxc_workspace_create
 *    (size from pxc_workspace_query).  A workspace is not thread-safe; use one
 *    workspace per concurrent stream.
 *  - Calls are asynchronous on `stream` and return a pxc_status describing the
 *    host-side checks and launch errors.  Errors found by the kernels (bad state
 *    id, non-finite input, exponent overflow, a bounded wait that ran out) are
 *    latched in the workspace and returned by pxc_sync_status (which
 *    synchronises the stream) or pxc_get_stats.  Results of a call that latched
 *    an error are unspecified.
 *  - No exception crosses the ABI.  pxc_last_error() gives a thread-local
 *    message for the last non-OK status returned on the calling thread.
 *  - Units: energies and wavenumbers in cm^-1, A in s^-1, T in K, P in bar,
 *    gamma_ref in cm^-1 per unit of P, mass in Da; intensities in cm/molecule,
 *    cross sections in cm^2/molecule.
 *  - State ids are 0-based and dense: transition t connects upper[t] and
 *    lower[t], both in [0, states.n).
 *  - Scaled results: intensities and cross sections are returned in FP32
 *    scaled by a per-list power of two, value = stored * 2^exp, so that lists
 *    whose lines are ~1e-50 neither underflow nor vanish.
 */
#ifndef PXC_H
#define PXC_H

#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PXC_OK = 0,
  PXC_ERR_ARG = 1,        /* null pointer, n < 0, dnu <= 0, T <= 0, cutoff < 0, ... */
  PXC_ERR_ID_RANGE = 2,   /* a state id outside [0, states.n) */
  PXC_ERR_NONFINITE = 3,  /* an infinite energy or a non-finite A */
  PXC_ERR_OVERFLOW = 4,   /* a Boltzmann exponent above 709.78 (negative energy at low T) */
  PXC_ERR_TIMEOUT = 5,    /* a bounded device wait ran out; the kernel returned early */
  PXC_ERR_CUDA = 6,       /* a CUDA launch or runtime error */
  PXC_ERR_CAPACITY = 7    /* the call exceeds the capacity the workspace was sized for */
} pxc_status;

/* States (Sec. 2.3, .states file): energy term values E, total degeneracies g,
 * and, for two-temperature non-LTE, the vibrational part E_vib of each energy
 * (Eq. Enonlte; E_rot = E - E_vib, Eq. Erot nonlte).  E_vib may be NULL for LTE.
 * A state whose E is NaN is absent: it adds nothing to Q and its lines are dropped. */
typedef struct {
  const double* E;       /* [n] cm^-1 */
  const int32_t* g;      /* [n] total degeneracy */
  const double* E_vib;   /* [n] cm^-1, or NULL */
  int64_t n;
  const double* n_vib;   /* [n] custom vibronic densities (Sec. 3.1.3, Eq. Nvib), or NULL: with
                            E_vib and a condition with T_vib <= 0, the populations are
                            g n_vib exp(-c2 (E - E_vib) / T_rot) (Eq. F nlte Nvib), T = T_rot,
                            Q by Eq. (Q nlte Nvib) and absorption by Eq. (nlte ab pop density).
                            A condition with T_vib > 0 and n_vib set is PXC_ERR_ARG. */
} pxc_states;

/* Transitions (Sec. 2.3, .trans file): upper id, lower id, Einstein A.
 * A is float64 unless A_is_f32 != 0 (then float32). */
typedef struct {
  const int32_t* upper;  /* [n] */
  const int32_t* lower;  /* [n] */
  const void* A;         /* [n] s^-1 */
  int32_t A_is_f32;
  int64_t n;
} pxc_transitions;

/* One thermodynamic condition.  T_vib <= 0 selects LTE at temperature T
 * (Eq. F lte); T_vib > 0 selects the two-temperature Treanor populations
 * (Eq. F nlte 2T) with T_rot = T, and T_rot then also sets the Doppler and
 * pressure widths (Sec. 3.3). */
typedef struct {
  double T;
  double T_vib;
  double P;              /* bar */
} pxc_condition;

/* Spectral grid (Sec. 2.4.3).  wl_unit == 0: wavenumbers nu_i = nu_min + i * dnu, i = 0 .. n-1.
 * wl_unit > 0: wavelengths lambda_i = nu_min + i * dnu (the fields then hold lambda_min and
 * dlambda) in the unit with nu = wl_unit / lambda: 1e7 for nm, 1e4 for um.  On a wavelength grid
 * sigma is sampled at nu_i = wl_unit / lambda_i, the cut-off stays in cm^-1, the window of a line
 * is i_lo = ceil((U/(nu + cut) - lambda_min)/dlambda), i_hi = floor((U/(nu - cut) - lambda_min)/
 * dlambda) (the last point when nu <= cut), lines are ordered by descending nu (ties by index),
 * and only the sampled kinds (0..3, 8..10) are accepted, forward only. */
typedef struct {
  double nu_min;
  double dnu;
  int64_t n;
  double wl_unit;
} pxc_grid;

/* Line profiles (Table profile). */
typedef enum {
  PXC_GAUSS_DOPPLER = 0, /* Doppler HWHM alpha = (nu/c) sqrt(2 N_A k_B T ln2 / M) */
  PXC_GAUSS_HWHM = 1,    /* Gaussian with the fixed HWHM `hwhm` */
  PXC_LORENTZ = 2,       /* gamma = gamma_ref (T_ref/T)^n_T P */
  PXC_VOIGT = 3,         /* Voigt of the Doppler alpha and the Lorentz gamma */
  /* Binned profiles (Table profile): the average of the profile over the grid bin
   * [nu_i - dnu/2, nu_i + dnu/2] centred on each point, so sum_i sigma_i dnu keeps the line
   * intensity on any grid (no undersampling loss).  Widths as the base kind (kind & 3).
   * Forward only (pxc_cross_section_backward returns PXC_ERR_ARG). */
  PXC_BINNED_GAUSS_DOPPLER = 4, /* erf / erfc differences */
  PXC_BINNED_GAUSS_HWHM = 5,
  PXC_BINNED_LORENTZ = 6,       /* arctangent difference */
  PXC_BINNED_VOIGT = 7,         /* composite 2-point Gauss-Legendre over the bin, subintervals of a
                                   quarter of the local width scale, at most 1024 per bin */
  /* Pseudo-Voigt approximations (Table profile): a Lorentzian and a Gaussian of one common full
   * width G, mixed with weights wL, wG, from the Voigt kind's Doppler and Lorentz widths (full
   * widths fG = 2 alpha, fL = 2 gamma).  Sampled, forward only. */
  PXC_PV_THOMPSON = 8,          /* Thompson, Cox, Hastings (1987): G from the fifth-power formula,
                                   wL = 1.36603 r - 0.47719 r^2 + 0.11116 r^3, r = fL / G */
  PXC_PV_OLIVERO = 9,           /* Olivero, Longbothum (1977) width G = 0.5346 fL + sqrt(0.2166 fL^2 + fG^2),
                                   the same mixing */
  PXC_PV_LIULIN = 10            /* Liu, Lin et al. (2001): width and both weights as cubic/analytic
                                   functions of d = (fL - fG)/(fL + fG); wL + wG differs from 1 by
                                   up to 0.73 % */
} pxc_profile;

typedef struct {
  int32_t kind;          /* pxc_profile */
  double cutoff;         /* line-wing cut-off: points with |nu_i - nu_l| <= cutoff */
  double mass_da;        /* molecular mass (Doppler widths) */
  double hwhm;           /* PXC_GAUSS_HWHM only */
  const float* gamma_ref;/* [transitions.n] (Lorentz, Voigt), else NULL */
  const float* n_T;      /* [transitions.n] temperature exponents (Lorentz, Voigt) */
  double T_ref;          /* reference temperature of gamma_ref, normally 296 K */
} pxc_profile_args;

/* Capacity a workspace is sized for. */
typedef struct {
  int64_t max_states;
  int64_t max_lines;       /* transitions per call (per chunk when streaming) */
  int64_t max_grid;
  int32_t max_conditions;  /* conditions per batched call */
  int32_t max_temperatures;/* distinct (T, T_vib) pairs per batched call; 0 means max_conditions */
} pxc_capacity;

typedef struct pxc_workspace pxc_workspace;

/* Bytes of device scratch a workspace of this capacity needs. */
pxc_status pxc_workspace_query(const pxc_capacity* cap, size_t* bytes);

/* Bind a workspace to `device_scratch` (device memory of at least the queried
 * size, 256-byte aligned, owned by the caller and kept alive until destroy).
 * The handle itself is host memory owned by the library. */
pxc_status pxc_workspace_create(const pxc_capacity* cap, void* device_scratch, size_t bytes,
                                pxc_workspace** ws);
pxc_status pxc_workspace_destroy(pxc_workspace* ws);

/* Synchronise `stream`, return and clear the latched device error. */
pxc_status pxc_sync_status(pxc_workspace* ws, cudaStream_t stream);

/* Thread-local message for the last non-OK status. */
const char* pxc_last_error(void);

/* Number of CUDA kernels this library has launched since it was loaded (all
 * workspaces and threads); differences around a region count its launches. */
int64_t pxc_kernel_launches(void);

/* Accumulate mode (streaming a line list in chunks, Sec. 2.1 and 4: bounded
 * memory over large .trans files).  When on, pxc_cross_section ADDS the chunk's
 * lines to sigma_out, whose current exponent is read from sigma_exp_out
 * (initialise it to PXC_EXP_EMPTY before the first chunk); if a chunk raises
 * the exponent the existing sum is rescaled on the device.  The partition
 * function is computed on the first chunk and reused while accumulating, so
 * the states must not change between chunks. */
#define PXC_EXP_EMPTY (-2147483647 - 1)
pxc_status pxc_set_accumulate(pxc_workspace* ws, int on);

/* Emission mode (Sec. 3.2, emission intensities).  When on, pxc_line_intensities,
 * pxc_cross_section and pxc_cross_section_streamed use emission intensities
 * epsilon = g' h c A nu p' / (4 pi Q) in erg/s/sr/molecule, p' the upper-state
 * population of the condition's model: Eq. (ems intensity lte), Eq. (nlte em 2T) or
 * Eq. (nlte em pop density).  sigma is then the emission cross section sum epsilon f
 * (erg/s/sr/molecule per cm^-1), with the same cut-off, threshold (on epsilon), sort and
 * exponent handling.  pxc_cross_section_backward is absorption-only (PXC_ERR_ARG here). */
pxc_status pxc_set_emission(pxc_workspace* ws, int on);

/* CUDA-graph replay of pxc_cross_section (Sec. 4.4: a batched (T, P) table is re-evaluated with
 * the same preprocessing; the many small launches of the intensity, sort and binning passes are
 * then replayed as one graph).  When on, each distinct call -- the same pointers, sizes,
 * conditions, grid, profile arguments, threshold and outputs, and the same workspace modes and
 * tile -- is captured into a CUDA graph the first time it is made and replayed by later identical
 * calls (the device data behind the pointers may change between calls; the graph reads it
 * afresh).  Up to 8 graphs are kept per workspace, the least recently used dropped first.  The
 * capture runs on a stream the workspace owns, so the caller's stream may be the legacy default
 * stream; the first call of a shape therefore costs a capture and an instantiation.  Accumulate
 * mode is never captured (its result depends on the workspace's running state), and pass timing
 * (pxc_set_timing) is not recorded for replays.  Turning graphs off frees the cached graphs.
 * No counterpart in the paper. */
pxc_status pxc_set_graphs(pxc_workspace* ws, int on);
/* Captures made, replays made and graphs cached by this workspace (each pointer nullable). */
pxc_status pxc_graph_stats(pxc_workspace* ws, int64_t* captures, int64_t* replays, int32_t* cached);

/* Bound, in SM clock cycles, of the profile kernel's waits for line records staged by bulk
 * copies (default 4e9, about 2 s).  A wait that runs out sets PXC_ERR_TIMEOUT (returned by
 * pxc_sync_status); its CTA lets the copies it issued land and returns, so the context and the
 * workspace stay usable.  A limit of 0 makes the waits give up at once: the failure path can be
 * exercised without any fault.  No counterpart in the paper.  PXC_ERR_ARG if cycles < 0. */
pxc_status pxc_set_wait_limit(pxc_workspace* ws, int64_t cycles);

/* Partition functions, Eq. (pf) (LTE) or Eq. (Q nlte 2T) (T_vib > 0), summed in
 * FP64 over all states for each of the n_c conditions.
 * Q_out:  [n_c] device.
 * dQ_out: [n_c][2] device, or NULL: dQ/dT (LTE) or dQ/dT_rot, and dQ/dT_vib.
 * Errors: PXC_ERR_OVERFLOW if some exponent exceeds 709.78, PXC_ERR_NONFINITE
 * for an infinite energy (latched). */
pxc_status pxc_partition_function(pxc_workspace* ws, const pxc_states* states,
                                  const pxc_condition* c, int32_t n_c,
                                  double* Q_out, double* dQ_out, cudaStream_t stream);

/* Stick spectrum (Sec. 2.4.3, "Stick spectra"): per transition t
 *   nu_out[t]       = E[upper] - E[lower] (FP64, bit-exact IEEE subtraction)
 *   I_scaled_out[t] = I_t * 2^-k in FP32, I_t by Eq. (abs intensity lte) or
 *                     Eq. (nlte ab 2T); 0 for dropped lines
 *   *I_exp_out      = k, the frexp exponent of the largest kept I (device int32)
 *   *n_kept_out     = number of kept lines (device int64)
 * A line is kept when nu > 0 (lines with negative centres are discarded,
 * Sec. 2.4.3), I >= threshold and, if grid != NULL, its cut-off window
 * [nu - cutoff, nu + cutoff] contains a grid point.
 * Any output pointer may be NULL except I_exp_out. */
pxc_status pxc_line_intensities(pxc_workspace* ws, const pxc_states* states,
                                const pxc_transitions* trans, const pxc_condition* c,
                                const pxc_grid* grid, double cutoff, double threshold,
                                double* nu_out, float* I_scaled_out, int32_t* I_exp_out,
                                int64_t* n_kept_out, cudaStream_t stream);

/* Cross sections, Eq. (xsec): sigma(nu_i) = sum_l I_l f_l(nu_i - nu_l) over the
 * kept lines with |nu_i - nu_l| <= cutoff, the truncated profile not renormalised.
 * The window of line l is i_lo = ceil((nu_l - cutoff - nu_min)/dnu),
 * i_hi = floor((nu_l + cutoff - nu_min)/dnu) in IEEE double.
 * For each condition j < n_c:
 *   sigma_out[j * grid.n + i] * 2^sigma_exp_out[j]  (FP32 scaled, exponent int32)
 * Lines are sorted exactly by (nu, index), binned into grid segments and
 * accumulated in FP32 with compensated stage sums; nu, the Boltzmann factors
 * and Q are FP64.  n_c > 1 evaluates the whole (T, P) table in one persistent
 * launch.  In accumulate mode n_c must be 1. */
pxc_status pxc_cross_section(pxc_workspace* ws, const pxc_states* states,
                             const pxc_transitions* trans, const pxc_condition* c, int32_t n_c,
                             const pxc_grid* grid, const pxc_profile_args* prof, double threshold,
                             float* sigma_out, int32_t* sigma_exp_out, cudaStream_t stream);

/* Adjoint of a scalar loss L(sigma_s) through pxc_cross_section for ONE
 * condition (n_c must be 1), given dL_dsigma = dL/dsigma_s on the grid, where
 * sigma_s is the scaled sigma_out the forward call returns (its exponent is
 * held constant).  Profiles are recomputed, not stored.  Outputs (device):
 *   dL_dT[0]         dL/dT (LTE) or dL/dT_rot (two-temperature)   FP64
 *   dL_dTvib[0]      dL/dT_vib (0 for LTE)                        FP64, nullable
 *   dL_dP[0]         dL/dP                                        FP64, nullable
 *   dL_dgamma_ref[t] per transition (0 for dropped lines)         FP32, nullable
 *   dL_dA[t]         per transition (0 for dropped lines)         FP32, nullable
 * Kept-line selection (threshold, window) is treated as fixed. */
pxc_status pxc_cross_section_backward(pxc_workspace* ws, const pxc_states* states,
                                      const pxc_transitions* trans, const pxc_condition* c, int32_t n_c,
                                      const pxc_grid* grid, const pxc_profile_args* prof, double threshold,
                                      const float* dL_dsigma, double* dL_dT, double* dL_dTvib,
                                      double* dL_dP, float* dL_dgamma_ref, float* dL_dA,
                                      cudaStream_t stream);

/* Reuse of the forward's line list by the adjoint (off by default).  When on, a single-condition
 * pxc_cross_section on a wavenumber grid (absorption, not in accumulate mode, a kind with an
 * adjoint) also keeps the sorted per-line ids and A the adjoint needs, and a following
 * pxc_cross_section_backward whose arguments (arrays, sizes, condition, grid, profile, threshold)
 * are identical to that call's skips the intensity pass, sort and preparation and reads the
 * forward's kept, sorted lines instead.  Any other call on the workspace in between (or this
 * call) discards the kept list.  The caller guarantees that the contents of the arrays have not
 * changed since the forward call (as an autograd forward/backward pair does); the backward's
 * results are then bit-identical to those without reuse. */
pxc_status pxc_set_reuse_forward(pxc_workspace* ws, int32_t on);

/* Diagnostics of the last pxc_cross_section / backward call on this workspace
 * (host values; synchronises the stream).  Counts are over the last condition. */
typedef struct {
  int64_t n_kept;          /* kept lines */
  int64_t n_nonzero;       /* kept lines whose FP32 scaled intensity is non-zero */
  int64_t evals_window;    /* sum over kept lines of their window size (algorithmic count) */
  int64_t evals_nonzero;   /* the same over kept lines with non-zero scaled intensity */
  int32_t segment_points;  /* grid points per segment used by the profile kernel */
  int32_t n_segments;
  int32_t I_exp;           /* exponent k of the last condition */
  int32_t tile;            /* profile tile configuration used (0 .. PXC_NUM_TILES-1) */
} pxc_stats;
pxc_status pxc_get_stats(pxc_workspace* ws, cudaStream_t stream, pxc_stats* out);

/* The sorted line order and segment binning of the last call (device outputs):
 * perm_out[j] = transition index of the j-th kept line in (nu bits, index)
 * order, j < n_kept; seg_first/seg_last [n_segments]: the lines whose windows
 * meet segment s are perm[seg_first[s] .. seg_last[s]-1].  Nullable. */
pxc_status pxc_get_binning(pxc_workspace* ws, int64_t* perm_out, int64_t* seg_first,
                           int64_t* seg_last, cudaStream_t stream);

/* Optional CUDA-event timing of the passes of pxc_cross_section on this
 * workspace (events recorded on the call's stream around each pass).
 * pxc_get_timing synchronises `stream` and returns, since the last read,
 * ms[0] intensity pass, ms[1] compaction + sort + preparation, ms[2] profile
 * pass, and count[i] the number of timed launches of each (count nullable). */
pxc_status pxc_set_timing(pxc_workspace* ws, int on);
pxc_status pxc_get_timing(pxc_workspace* ws, cudaStream_t stream, double* ms, int64_t* count);

/* Profile-kernel tile configurations.  The profile pass (Eq. xsec summed over
 * the kept lines) splits the grid into segments of S points, one work item per
 * segment and line range.  The compiled configurations are
 *   tile 0: S = 128  (32 threads x 4 points, 64 lines per stage)
 *   tile 1: S = 256  (64 threads x 4 points, 64 lines per stage)
 *   tile 2: S = 1024 (128 threads x 8 points, 64 lines per stage)
 *   tile 3: S = 2048 (128 threads x 16 points, 128 lines per stage)
 * and every one gives the same sigma up to FP32 summation order.  Wavelength grids always
 * use 128-point segments.  The workspace
 * keeps one tile per profile kind for single-condition calls (batched = 0,
 * default tile 0) and one for batched tables (batched = 1, default tile 0). */
#define PXC_NUM_TILES 4
pxc_status pxc_set_tile(pxc_workspace* ws, int32_t kind, int32_t batched, int32_t tile);
pxc_status pxc_get_tile(pxc_workspace* ws, int32_t kind, int32_t batched, int32_t* tile);

/* Autotuner: runs pxc_cross_section with every tile configuration on the
 * caller's own inputs (same arguments as pxc_cross_section), `repeats` timed
 * runs each after one warm-up run, times each run with CUDA events on
 * `stream`, and keeps the fastest tile in the workspace for this profile kind
 * and for single (n_c == 1) or batched (n_c > 1) calls.  ms_out [PXC_NUM_TILES]
 * (host, nullable) receives each tile's mean milliseconds per call; *tile_out
 * (host, nullable) the tile chosen.  sigma_out / sigma_exp_out end holding the
 * result of the chosen tile.  Synchronises `stream`. */
pxc_status pxc_autotune(pxc_workspace* ws, const pxc_states* states, const pxc_transitions* trans,
                        const pxc_condition* c, int32_t n_c, const pxc_grid* grid,
                        const pxc_profile_args* prof, double threshold, float* sigma_out,
                        int32_t* sigma_exp_out, int32_t repeats, int32_t* tile_out, double* ms_out,
                        cudaStream_t stream);

/* Stream a HOST-resident line list through the device in chunks of
 * cap.max_lines transitions (Sec. 2.1: bounded-memory streaming of large
 * .trans files; Sec. 4.4: one preprocessing pass reused for every output).
 * Host arrays should be pinned for overlap.  States are device-resident.
 * Copies of chunk i+1 overlap the kernels of chunk i (two device staging
 * buffers of dev_chunk_bytes each, caller-owned, from pxc_stream_buffer_bytes).
 * Result: sigma_out (device) * 2^(*sigma_exp_out) (device int32). */
size_t pxc_stream_buffer_bytes(int64_t chunk_lines, int32_t A_is_f32, int32_t with_broadening);
pxc_status pxc_cross_section_streamed(pxc_workspace* ws, const pxc_states* states,
                                      const int32_t* host_upper, const int32_t* host_lower,
                                      const void* host_A, int32_t A_is_f32,
                                      const float* host_gamma_ref, const float* host_n_T,
                                      int64_t n_lines, const pxc_condition* c,
                                      const pxc_grid* grid, const pxc_profile_args* prof, double threshold,
                                      void* dev_chunk_buf0, void* dev_chunk_buf1, size_t dev_chunk_bytes,
                                      float* sigma_out, int32_t* sigma_exp_out, cudaStream_t stream);

/* Cooling functions, Eq. (cf): W = sum over transitions with nu = E' - E'' > 0 of
 * g' h c A nu p' / (4 pi Q), in erg/s/sr/molecule, for each of n_c conditions (p' and Q
 * of the condition's population model: LTE, two-temperature or vibronic densities;
 * no grid window and no threshold).  W_out [n_c] device; Q_out [n_c] device or NULL.
 * Computed as W = (h c / 4 pi Q) sum_s g_s p_s S_s with S_s = sum over lines leaving
 * state s of A nu: one pass over the lines (FP64 atomic adds, so the last bits depend
 * on their order) and one pass over the states per condition.  Needs max_conditions
 * >= n_c.  Errors as pxc_partition_function, plus PXC_ERR_ID_RANGE and
 * PXC_ERR_NONFINITE (latched) for bad ids or A. */
pxc_status pxc_cooling_function(pxc_workspace* ws, const pxc_states* states, const pxc_transitions* trans,
                                const pxc_condition* c, int32_t n_c, double* W_out, double* Q_out,
                                cudaStream_t stream);

/* Partition functions for callers that cannot allocate device memory.
 * No counterpart in the paper: this is a deployment variant of
 * pxc_partition_function for code that may not call cudaMalloc at all (a
 * plug-in inside an application that owns all device memory, a real-time path
 * that cannot afford cudaMalloc's device-wide synchronisation, a caller with
 * nowhere to keep a workspace).  It takes no workspace and allocates nothing:
 * its scratch is a fixed ~1.8 MB array inside the library that every device
 * loading the library keeps until the process exits.
 *   n_c <= 64 conditions (PXC_ERR_CAPACITY otherwise); Q_out [n_c] and
 *   dQ_out [n_c][2] (nullable) as in pxc_partition_function; status_out
 *   (device int32, nullable) receives PXC_OK, PXC_ERR_NONFINITE or
 *   PXC_ERR_OVERFLOW once the kernels have run.
 * All calls share that array: calls overlapping on the GPU (several streams or
 * host threads) race and must be serialised.  The first call on a device looks
 * up the array's address with that device current; make it before any stream
 * capture. */
pxc_status pxc_partition_function_noalloc(const pxc_states* states, const pxc_condition* c, int32_t n_c,
                                          double* Q_out, double* dQ_out, int32_t* status_out,
                                          cudaStream_t stream);

/* Instruction-throughput microbenchmark of the current device (no counterpart in the paper;
 * the profile pass of Eq. xsec is bound by these pipes, so its roofline is stated against
 * rates measured on the chip).  Runs one full wave of four kernels on `stream` and synchronises:
 *   host_out[0] FP32 FMA results per SM per clock cycle
 *   host_out[1] MUFU reciprocal (rcp.approx.ftz.f32) results per SM per clock cycle
 *   host_out[2] MUFU exp2 (ex2.approx.ftz.f32) results per SM per clock cycle
 *   host_out[3] far-wing Voigt evaluations (5 FP32 FMAs + 1 reciprocal each) per SM per clock
 *   host_out[4..7] the same four rates per second at the clock the device ran (CUDA events).
 * Per-clock rates come from the SM cycle counter of every CTA, so they do not depend on the
 * clock frequency.  dev_buf: caller device memory of pxc_pipe_rates_buffer_bytes() bytes.
 * PXC_ERR_ARG for a null or short buffer, PXC_ERR_CUDA if a kernel fails. */
size_t pxc_pipe_rates_buffer_bytes(void);
pxc_status pxc_pipe_rates(void* dev_buf, size_t bytes, double* host_out, cudaStream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* PXC_H */
