/*
 * fdtd.h -- C ABI of the GB300 time-reversible FDTD gradient library.
 *
 * The library computes L(eps) = sum_n l_n and dL/d(eps_r) for a 3D Yee FDTD
 * with a convolutional PML, using the time-reversible gradient of the paper
 * (Sec. 1-2): the forward run records only the fields on the interface
 * slices between the simulation volume and the PML, compressed by reduced
 * bit-width and by keeping every k-th step; the backward run reverses the
 * lossless interior in time, injects the recorded slices back (interpolated
 * in time) and runs the adjoint alongside.
 *
 * Units: normalised fields E and Ht = eta0 H; S = c dt / dx (Eq. 1 with
 * C = 0.99 gives S = 0.99/sqrt(3)).  Arrays are float32 [nz][ny][nx], x
 * fastest, contiguous.  Grid cells [P, N-P) along every axis form the
 * interior; the design box must lie inside it.
 *
 * Memory: the caller owns every device buffer (eps, gradient, workspace) and
 * the CUDA stream; the library never calls cudaMalloc.  Calls return an
 * fdtd_status and never throw; fdtd_last_error() gives a message.  One
 * handle must not be used from two threads at once.
 */
#ifndef FDTD_GB300_H
#define FDTD_GB300_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FDTD_ABI_VERSION 1

typedef enum {
  FDTD_OK = 0,
  FDTD_EINVAL = -1,     /* bad argument (message in fdtd_last_error) */
  FDTD_ENOMEM = -2,     /* workspace missing or too small; host allocation failed */
  FDTD_ECUDA = -3,      /* a CUDA runtime call failed */
  FDTD_ESTATE = -4,     /* call out of order (e.g. backward without forward) */
  FDTD_ETIMEOUT = -5,   /* a bounded device wait gave up */
  FDTD_ENONFINITE = -6  /* eps < 1 or non-finite, or a non-finite result */
} fdtd_status;

typedef struct fdtd_handle fdtd_handle;

typedef struct { int nx, ny, nz; } fdtd_grid;

/* Convolutional PML (Roden & Gedney, cited in Sec. 1) on all six faces.
 * Grading over the depth d in (0,1] from the interface:
 *   sigma dt/eps0 = sigma_factor (order+1) S d^order,
 *   kappa = 1 + (kappa_max-1) d^order,
 *   alpha dt/eps0 = alpha_factor 2 pi f0 dt (1-d),  f0 = c / lambda0.
 * Zero or negative fields select the defaults 3 / 0.8 / 1 / 0.05. */
typedef struct {
  int thickness;          /* P >= 1 cells */
  int order;
  double sigma_factor;
  double kappa_max;
  double alpha_factor;
} fdtd_pml;

enum { FDTD_SRC_NONE = 0, FDTD_SRC_POINT = 1, FDTD_SRC_PLANE_GAUSS = 2,
       FDTD_SRC_PLANE_UNIFORM = 3 };

/* Current source J entering E += (S/eps)(curl Ht - J).
 * J^{n+1/2} = amplitude w(u,v) g((n+1/2) dt),
 * g(t) = exp(-((t-t0)/tau)^2) sin(w0 (t-t0)), w0 = 2 pi c / lambda0,
 * tau = 2 sqrt(2 ln 2) / (rel_bandwidth w0) (power-spectrum FWHM),
 * t0 = t0_over_tau tau.
 * POINT: w = 1 at pos.  PLANE_GAUSS: plane normal `axis` at pos[axis];
 * w = exp(-(u-pos_u)^2/(2 su^2) - (v-pos_v)^2/(2 sv^2)) over the interior
 * cross-section, (u,v) the other two axes in increasing order.
 * PLANE_UNIFORM: the same plane with w = 1 over the interior cross-section,
 * a normally incident plane wave (the paper's coupler source, Sec. 4);
 * sigma_uv is ignored. */
typedef struct {
  int kind;
  int component;          /* 0..2 = Ex, Ey, Ez */
  int pos[3];
  int axis;
  double sigma_uv[2];
  double lambda0;         /* metres */
  double rel_bandwidth;
  double t0_over_tau;
  double amplitude;
} fdtd_source;

enum { FDTD_OBJ_E2_PLANE = 1, FDTD_OBJ_POYNTING_PLANE = 2 };

/* Objective l_n on the plane normal `axis` at `index`, cells (u,v) in
 * [lo,hi) with (u,v) the other two axes in increasing order:
 *   E2_PLANE:       l_n = sum |E^{n+1}|^2
 *   POYNTING_PLANE: l_n = sum (E^{n+1} x Ht^{n+1/2}) . axis
 * (components co-indexed at each cell; the Poynting detector stands for
 * the paper's flux detectors, Sec. 3). */
typedef struct {
  int kind;
  int axis;
  int index;
  int lo[2];
  int hi[2];
} fdtd_detector;

/* Tape element types.  E4M3 is the OCP / hardware float8 e4m3fn (max 448).
 * 4..8 are the 8-bit formats compared in Sec. 4 (Fig. 3), coded in software
 * (exponent bits, mantissa bits, bias, largest finite value):
 *   E4M3B11FNUZ 4,3,11, 30      E5M2FNUZ 5,2,16, 57344     E4M3FNUZ 4,3,8, 240
 *   E4M3_IEEE   4,3,7,  240     E3M4     3,4,3,  15.5
 * "fnuz": no infinities, no negative zero, NaN = 0x80; the IEEE-like ones
 * reserve the all-ones exponent for infinities and NaNs.  All encodings round
 * to nearest, ties to even, and saturate to the largest finite value.
 *
 * BDCT (9) is a block-transform codec beyond the paper (its Sec. 4 names
 * JPEG-like compression of the tape as future work): every face component
 * [v][u] is cut into 8 x 8 blocks (cells past the face edge repeat the last
 * row / column), each block is transformed with the orthonormal 2D DCT-II,
 * and the first `coeffs` coefficients in diagonal order (u + v ascending,
 * then v ascending) are kept as int8 codes round(C / s), s = max(max|C| /
 * 127, 2^-126) (1 for an all-zero block), with s stored as float32 per block.
 * All of it in float32 with a fixed operation order (fmaf over the block's
 * cells row by row, then over the kept coefficients in order), so that an
 * independent implementation reproduces the codes bit for bit. */
enum {
  FDTD_TAPE_F32 = 0, FDTD_TAPE_BF16 = 1, FDTD_TAPE_F16 = 2, FDTD_TAPE_E4M3 = 3,
  FDTD_TAPE_E4M3B11FNUZ = 4, FDTD_TAPE_E5M2FNUZ = 5, FDTD_TAPE_E4M3FNUZ = 6,
  FDTD_TAPE_E4M3_IEEE = 7, FDTD_TAPE_E3M4 = 8, FDTD_TAPE_BDCT = 9
};
enum { FDTD_INTERP_LINEAR = 0, FDTD_INTERP_CUBIC = 1 };

/* Boundary-tape compression (Sec. 2): storage type of the recorded slices,
 * k = keep every k-th step (the last step is always kept), and the time
 * interpolation used to restore the steps in between.  scaled = 1 stores a
 * per-face, per-sample FP32 scale max(absmax/format_max, 2^-126) (1 when the
 * face is all zero; F16 and the 8-bit types only); values are converted back
 * to FP32 before any arithmetic.  coeffs: BDCT only, coefficients kept per
 * 8 x 8 block (1..64; 0 = 10, the diagonals u + v <= 3); must be 0 for the
 * other types.  A BDCT sample holds int8 codes [face][comp][block][coeffs]
 * (zero-padded to 16 bytes), then float32 scales [face][comp][block]. */
typedef struct {
  int dtype;
  int k;
  int interp;
  int scaled;
  int coeffs;
} fdtd_record_cfg;

/* Plan a problem (Sec. 2, Fig. 2: a simulation volume surrounded by PML on
 * every face, a source, a detector and a design region; the time step obeys
 * the CFL bound of Eq. 1).  Host only: touches no device.  dx in metres, dt
 * in seconds with c dt / dx <= 1/sqrt(3).  n_steps >= 1.  design box
 * [lo, hi) inside the interior.  cuda_stream: the caller's stream (NULL =
 * legacy default stream); all work is ordered after work already queued
 * there, and later work queued there sees the results.
 * Errors: FDTD_EINVAL (message in fdtd_last_error(NULL)), FDTD_ENOMEM. */
int fdtd_create(const fdtd_grid* grid, double dx, double dt, const fdtd_pml* pml,
                const fdtd_source* source, const fdtd_detector* detector, int n_steps,
                const int design_lo[3], const int design_hi[3], void* cuda_stream,
                fdtd_handle** out);

/* Bytes of device workspace needed for forward + backward with `rec`. */
int fdtd_workspace_bytes(const fdtd_handle* h, const fdtd_record_cfg* rec, size_t* bytes);

/* Bind caller-owned device memory (256-byte aligned) as the workspace.
 * It must stay valid until the handle is destroyed or rebound. */
int fdtd_bind_workspace(fdtd_handle* h, void* dptr, size_t bytes);

/* Bytes of the compressed boundary tape alone (samples + scales). */
int fdtd_tape_bytes(const fdtd_handle* h, const fdtd_record_cfg* rec, size_t* bytes);

/* Forward run (Sec. 2: the forward simulation records the field values at
 * the interface slices between the simulation volume and the PML, converted
 * to the tape's bit-width and kept every k-th step): n_steps leapfrog steps
 * from zero fields with eps (device, float32 [nz][ny][nx], every value
 * finite and >= 1), recording the boundary tape; writes L to *objective
 * (host).  Blocks until done.  Keeps the final state for fdtd_backward. */
int fdtd_forward(fdtd_handle* h, const float* d_eps, const fdtd_record_cfg* rec,
                 double* objective);

/* Backward run (Sec. 2: the time-reversed simulation, with the recorded
 * values converted back to float32, interpolated in time and injected at
 * the interface slices, which act as sources; the adjoint runs alongside and
 * gives the gradient, Sec. 1): seed * dL/d(eps) over the design box into
 * d_grad_eps (device, float32 [dz][dy][dx]).  Needs a preceding
 * fdtd_forward; consumes its state (FDTD_ESTATE otherwise).  Blocks until
 * done. */
int fdtd_backward(fdtd_handle* h, double seed, float* d_grad_eps);

/* Both directions with HOST buffers (end-to-end path): copies h_eps to the
 * device, runs forward and backward, copies seed * dL/d(eps) over the
 * design box to h_grad.  Pinned host memory makes the copies asynchronous. */
int fdtd_value_and_grad_host(fdtd_handle* h, const float* h_eps, const fdtd_record_cfg* rec,
                             double seed, double* objective, float* h_grad);

/* Batched designs: n independent handles (each with its own workspace)
 * processed together; objs[i] / d_grads[i] as in fdtd_forward/backward.
 * Each handle runs its own time loop (a CUDA graph on its own stream); all
 * are enqueued before any is awaited, so they run concurrently. */
int fdtd_group_forward(fdtd_handle* const* hs, int n, const float* const* d_eps,
                       const fdtd_record_cfg* rec, double* objs);
int fdtd_group_backward(fdtd_handle* const* hs, int n, const double* seeds,
                        float* const* d_grads);

/* Batched designs in one launch per half-step: the same results as the
 * group calls (fields and gradients equal to each handle's own run; the
 * objectives to the order of their FP64 sums), but every forward half-step
 * of every design runs as ONE launch over a list of (design, tile, z chunk)
 * units, and likewise the record, the restore and the reverse phases, each
 * CTA reading its design's own arguments and tensor maps from tables in
 * device memory.  Designs are taken in descending order of step count: at
 * forward step s (reverse iteration t) the designs with more than s (t)
 * steps run, design d at its step s (N_d - 1 - t).  The loops are captured
 * once into CUDA graphs; the plan (tables and graphs, allocated by the
 * library with cudaMalloc, outside the time loops) belongs to hs[0] and is
 * rebuilt when the list, a workspace or an option changes; it is freed with
 * hs[0].  Every handle must run kernel 5's split steps (FDTD_OPT_FORWARD and
 * FDTD_OPT_REVERSE resolving to 1) with 32 x 8 tiles and two stages, one
 * detector, no exact reversal, and an unscaled tape format; else
 * FDTD_EINVAL.  fdtd_batch_backward needs the handles' forwards to come
 * from one fdtd_batch_forward (or with one record config). */
int fdtd_batch_forward(fdtd_handle* const* hs, int n, const float* const* d_eps,
                       const fdtd_record_cfg* rec, double* objs);
int fdtd_batch_backward(fdtd_handle* const* hs, int n, const double* seeds,
                        float* const* d_grads);

/* Last error message of h, or of the last failed fdtd_create when h is NULL. */
const char* fdtd_last_error(const fdtd_handle* h);

/* Release host resources and CUDA objects (not the caller's memory). */
int fdtd_destroy(fdtd_handle* h);

/* ------------------------------------------------- second detector --- */

/* Attach a second detector plane (NULL or kind 0 detaches it), e.g. the
 * input-side flux of a transmission ratio (Sec. 4 measures the Poynting flux
 * above the coupler and in its output waveguide).  Its objective
 * M = sum_n m_n accumulates in each forward alongside L (one extra launch per
 * step).  Same validation as the create detector (FDTD_EINVAL).  Host only;
 * invalidates a pending forward. */
int fdtd_set_detector2(fdtd_handle* h, const fdtd_detector* detector2);
/* L and M of the last forward (M = 0 without a second detector).
 * FDTD_ESTATE before the first forward. */
int fdtd_objectives(const fdtd_handle* h, double* L, double* M);
/* Backward for the objective seed * L + seed2 * M: d_grad_eps receives
 * d(seed L + seed2 M)/d(eps) over the design box (one time-reversed run; the
 * seeds enter as the detectors' adjoint sources).  seed2 != 0 without a
 * second detector: FDTD_ESTATE.  Otherwise as fdtd_backward. */
int fdtd_backward2(fdtd_handle* h, double seed, double seed2, float* d_grad_eps);

/* ------------------------------------------------ tuning and timing --- */

enum {
  FDTD_OPT_USE_GRAPHS = 0,    /* 1 (default): replay the time loop as a CUDA graph */
  FDTD_OPT_KERNEL = 1,        /* 5 (default): half-steps that stage one z plane per iteration
                                 in shared memory with TMA box loads (two x-cells per thread,
                                 tile height at least 2); 0: the same half-steps with plain
                                 global loads, one cell per thread (an independent
                                 cross-check; the tiling, staging and z-group options do not
                                 apply to it).  Other values: FDTD_EINVAL */
  FDTD_OPT_TILE_Y = 2,        /* CTA tile height in cells (1, 2, 4, 8 default, 16); width 32 */
  FDTD_OPT_ZCHUNK = 3,        /* z planes per CTA (0 = whole column) */
  FDTD_OPT_SAMPLE_EVERY = 4,  /* m > 0: every m-th launch of a time loop opens a timed
                                 interval (CUDA events on the library's stream), see
                                 fdtd_kernel_timing (0 = off) */
  FDTD_OPT_STAGES = 6,          /* kernel 5: planes staged per CTA (2
                                   default, 3, 4): stages - 1 planes are in flight while one
                                   is computed */
  FDTD_OPT_PDL = 7,             /* kernel 5: 1 = launch as a programmatic dependent of the
                                   previous kernel (its launch and prologue overlap the
                                   previous kernel's tail); 0 (default) = plain stream order */
  FDTD_OPT_PREFETCH = 8,        /* kernel 5: 1 = when a plane is staged, warm L2 with the
                                   next plane's boxes; 0 (default) = off */
  FDTD_OPT_TILE_X = 9,          /* kernel 5 with tile height 8 and 2 or 3 stages: tile width
                                   32 (default) or 40 cells */
  FDTD_OPT_COMPACT_AUX = 10,    /* kernel 5: 1 (default) = its CPML auxiliaries are
                                   stored for the slab cells only (per axis, where the grid
                                   is long enough); 0 = full-grid arrays */
  FDTD_OPT_EXACT_REVERSAL = 11, /* kernel 5: q in 8..30 rounds every field increment of the
                                   leapfrog to a multiple of 2^-q, so that the fields stay on
                                   that grid and, while |E|, |Ht| < 2^(24-q), every float32
                                   update is exact and the time-reversed interior retraces
                                   the forward run bit for bit (with an FP32 k = 1 tape);
                                   0 (default) = plain float32 increments.  Other kernels
                                   or tile shapes than kernel 5's defaults (32 x 8 tiles,
                                   2 stages) with q != 0: FDTD_EINVAL at fdtd_forward */
  FDTD_OPT_ZCHUNK_FWD = 12,     /* kernel 5: z planes per CTA of the forward half-steps
                                   (0 = the whole column; -1, the default: FDTD_OPT_ZCHUNK
                                   when the forward runs in z groups, as it does by default;
                                   with one launch per half-step, 16 when that grid of CTAs
                                   fits in about one wave of resident CTAs, else
                                   FDTD_OPT_ZCHUNK); FDTD_OPT_ZCHUNK sets the reverse phases
                                   (and every other kernel) */
  FDTD_OPT_ZGROUPS = 13,        /* kernel 5: G in 0..16; G > 1 splits every half-step launch
                                   into G launches over consecutive ranges of its z chunks,
                                   each on its own stream and waiting only for the
                                   neighbouring ranges of the half-step before, so that
                                   one half-step's tail overlaps the next one's start
                                   (tape, restore and monitor launches join all ranges);
                                   results are unchanged.  0 (default) = automatic: 4 in
                                   the forward, 3 in the reverse; 1 = one launch per
                                   half-step.  Sampled kernel timing
                                   (FDTD_OPT_SAMPLE_EVERY) records only loops that run
                                   with one launch per half-step; the no-allocation entry
                                   point always runs that way */
  FDTD_OPT_INJECT_WAIT_TIMEOUT = 14, /* failure-detection test hook: L > 0 makes every backward
                                   (fdtd_backward, fdtd_backward2, the group and no-allocation
                                   calls) start with one bounded device wait that nothing
                                   completes; it gives up after L SM cycles and sets the
                                   timeout bit of the device error word, so the call returns
                                   FDTD_ETIMEOUT with the CUDA context usable.  0 (default) =
                                   off.  Injects no fault: the wait is the same bounded wait
                                   as fdtd_selftest_wait */
  FDTD_OPT_REVERSE = 15,        /* kernel 5: how a reverse time step runs.  0 (default) =
                                   automatic: fused with 32 x 8 tiles when at most half of
                                   the (tile, z chunk) units carry CPML terms (see
                                   fdtd_reverse_units), else split; 1 = split:
                                   a reverse E phase and a reverse H phase, each updating the
                                   primal and the adjoint fields in place; 2 = fused: one
                                   launch for the primal fields (both inverse half-steps,
                                   interior cells, with dL/d(eps) accumulated) and one for the
                                   adjoint fields (both transposed half-steps, every cell),
                                   each reading every field once and writing it once into
                                   the other buffer of a ping-pong pair (the workspace holds
                                   a second field and adjoint buffer); FDTD_EINVAL at
                                   fdtd_forward with other tiles.  Results agree with the
                                   split phases: primal fields bit for bit, gradients to
                                   rounding */
  FDTD_OPT_FORWARD = 16,        /* kernel 5: how a forward time step runs.  0 (default) =
                                   automatic: where at most half of the (tile, z chunk)
                                   units carry CPML terms, two steps per pass (3) where it
                                   can run (below), else fused where it can run; split
                                   elsewhere; 1 = split: an H and an E half-step launch, each
                                   updating the fields in place; 2 = fused: the units
                                   without a CPML term (fdtd_reverse_units' CPML-free box)
                                   run both half-steps in one launch that reads every field
                                   once and writes it once into the other buffer of a
                                   ping-pong pair, and the other units run the split
                                   half-steps from and into the same pair.  Needs 32 x 8
                                   tiles, such units, and the source and the detector
                                   outside them; else FDTD_EINVAL at fdtd_forward.  The
                                   fields are bit-identical to the split half-steps'; 3 =
                                   two steps per pass (temporal blocking, not part of the
                                   paper's method): the deep units (fdtd_deep_units: no
                                   CPML term on their cells or a two-cell halo) run time
                                   steps n and n + 1 in one launch that reads E^n,
                                   Ht^{n-1/2} and cb once and writes E^{n+2}, Ht^{n+3/2}
                                   once into the other buffer of the pair, plus the
                                   intermediate level on the one-cell frame of the deep
                                   box into a third field buffer; the other units run the
                                   split half-steps one step at a time through that
                                   buffer.  Needs 32 x 8 tiles, deep units, and the source
                                   and the detectors two cells or more away from them;
                                   else FDTD_EINVAL at fdtd_forward.  An odd step count
                                   runs its first step as split half-steps over every
                                   unit.  The fields and the tape are bit-identical to
                                   the split half-steps' */
  FDTD_OPT_ZCHUNK_FWD2 = 17     /* kernel 5 with FDTD_OPT_FORWARD = 3: z planes per CTA of
                                   the two-step pass (-1 or 0, the default: sixteen chunks
                                   of the other units' split half-steps, whose chunks are
                                   FDTD_OPT_ZCHUNK_FWD planes if > 0, else FDTD_OPT_ZCHUNK);
                                   a chunk streams two planes below and one above it */
};
int fdtd_set_option(fdtd_handle* h, int option, int value);
int fdtd_get_option(const fdtd_handle* h, int option, int* value);

/* Kernel kinds for fdtd_kernel_timing. */
enum {
  FDTD_K_FWD_H = 0, FDTD_K_FWD_E = 1, FDTD_K_RECORD = 2, FDTD_K_RESTORE = 3,
  FDTD_K_REV_E = 4, FDTD_K_REV_H = 5, FDTD_K_REV_PRIMAL = 6, FDTD_K_REV_ADJOINT = 7,
  FDTD_K_MONITOR = 8, FDTD_K_REV_ADJOINT_CPML = 9, FDTD_K_FWD_FUSED = 10,
  FDTD_K_FWD_2STEP = 11, FDTD_K_KINDS = 12
};
/* Average in-loop cost (ms) per launch of one kernel kind in the last
 * forward + backward, and the number of samples it rests on
 * (FDTD_OPT_SAMPLE_EVERY = m must be > 0).  Every m-th launch opens an
 * interval timed with CUDA events, alternately around one launch (kind p)
 * and around two consecutive launches (kind p, then kind q); the cost of q is
 * mean(pair p->q) - mean(single p), so the events' own overhead cancels and
 * the result is q's duration plus its launch gap after p.  0 when a kind was
 * not sampled. */
int fdtd_kernel_timing(const fdtd_handle* h, int kind, float* avg_ms, int* samples);

/* Device time (CUDA events on the library's stream) of the last forward
 * time loop and backward time loop, in milliseconds, and the number of
 * kernel launches each issued. */
int fdtd_last_timing(const fdtd_handle* h, float* fwd_ms, float* bwd_ms, int* fwd_launches,
                     int* bwd_launches);

/* Device time (CUDA events on the library's stream, milliseconds) of the
 * last successful fdtd_value_and_grad_host between the end of its input
 * copy and the start of its output copy: eps -> cb, the forward and
 * backward time loops, the host waits between them and the gradient
 * finalisation; 0 before the first such call. */
int fdtd_last_host_call_ms(const fdtd_handle* h, float* device_ms);

/* ------------------------------------------------ introspection --------- */

/* Host copies of the plan's tables (no device needed).  which: 0 b_E,
 * 1 a_E, 2 1/kappa_E (integer positions), 3 b_H, 4 a_H, 5 1/kappa_H
 * (half-integer positions); out has the axis length. */
int fdtd_pml_profile(const fdtd_handle* h, int axis, int which, float* out);
/* J waveform amplitude * g((n+1/2) dt) for n = 0..n_steps-1. */
int fdtd_source_waveform(const fdtd_handle* h, float* out);
/* Interpolation of reverse step `step`: field 0 = Ht^{step+1/2} on the low
 * faces, 1 = E^{step} on the high faces.  Writes 4 (slot, weight) pairs;
 * slot -1 marks an unused entry (or the known zero initial state). */
int fdtd_interp_weights(const fdtd_handle* h, const fdtd_record_cfg* rec, int step, int field,
                        int* slot, float* weight);

/* Checkpoint of a forward run (the state fdtd_backward consumes): the final
 * fields, the coefficients cb, the boundary tape with its scales and the
 * per-step objectives, with a header naming the problem and record config.
 * fdtd_state_bytes: size of the blob for the last forward (host only;
 * FDTD_ESTATE without one).  fdtd_save_state: copies it into host memory
 * (bytes >= fdtd_state_bytes, else FDTD_EINVAL); the handle keeps its state.
 * fdtd_load_state: makes a handle of the same problem (grid, PML, steps,
 * second detector) ready for fdtd_backward as if it had run that forward;
 * its bound workspace must fit the saved record config.  Errors: FDTD_EINVAL
 * for a blob of another problem or a bad header, FDTD_ESTATE without a
 * workspace, FDTD_ENOMEM if it is too small. */
int fdtd_state_bytes(const fdtd_handle* h, size_t* bytes);
int fdtd_save_state(fdtd_handle* h, void* host_buf, size_t bytes);
int fdtd_load_state(fdtd_handle* h, const void* host_buf, size_t bytes);

/* Copy the current E, Ht (6 x [nz][ny][nx] float32) into d_out (device). */
int fdtd_read_fields(fdtd_handle* h, float* d_out);
/* Per-step objective l_n of the last forward (host, n_steps doubles). */
int fdtd_objective_history(fdtd_handle* h, double* out);

/* Tape codec on raw device arrays, for tests: encode n float32 values with
 * one scale (absmax/format_max when scaled, else 1) written to *d_scale,
 * and decode them back.  d_code holds n elements of the tape type. */
int fdtd_encode(int dtype, int scaled, const float* d_in, size_t n, void* d_code, float* d_scale,
                void* cuda_stream);
int fdtd_decode(int dtype, const void* d_code, size_t n, const float* d_scale, float* d_out,
                void* cuda_stream);

/* BDCT codec on one raw device plane, for tests: d_in float32 [nv][nu]
 * (nu, nv >= 1) -> d_codes int8 [nblocks][coeffs] and d_scales float32
 * [nblocks], nblocks = ceil(nu/8) ceil(nv/8) in row-major block order; decode
 * writes the reconstructed [nv][nu] plane.  coeffs in 1..64 (FDTD_EINVAL
 * otherwise).  Asynchronous on cuda_stream. */
int fdtd_bdct_encode(const float* d_in, int nu, int nv, int coeffs, signed char* d_codes,
                     float* d_scales, void* cuda_stream);
int fdtd_bdct_decode(const signed char* d_codes, const float* d_scales, int nu, int nv, int coeffs,
                     float* d_out, void* cuda_stream);
/* The BDCT basis table (host, no device use): out[i*64 + y*8 + x] = the
 * float32 value of basis function i (diagonal order) at cell (x, y).  The
 * first BDCT use on a device uploads this table synchronously, so it must
 * not happen while the caller's stream is being captured. */
int fdtd_bdct_basis(float* out);

/* The z-chunk ranges of the z-group schedule (FDTD_OPT_ZGROUPS; host only,
 * no device use): nch >= 1 z chunks split into min(G, nch) groups, G >= 1;
 * group g covers chunks [lo[g], hi[g]) (lo, hi: caller arrays of at least
 * min(G, nch) ints).  Returns the group count, or FDTD_EINVAL.  In the
 * schedule, group g of a half-step waits for groups g - 1 and g + 1 of the
 * half-step before (and for its own through stream order). */
int fdtd_zgroup_ranges(int nch, int G, int* lo, int* hi);

/* The (tile x, tile y, z chunk) units of the three launches of a fused
 * reverse step (FDTD_OPT_REVERSE), 32 x 8 tiles and zchunk planes (0 = the
 * whole column) on an nx x ny x nz grid with P CPML cells (host only, no
 * device use).  counts[0..2] receive the unit counts of the primal launch
 * (every unit with an interior cell), of the adjoint launch without CPML
 * terms (units whose cells and neighbours x0-1 .. x0+32, y0-1 .. y0+8, planes
 * k0-1 .. k1 are all interior) and of the adjoint launch with CPML (all other
 * units).  With units != NULL the units follow as int triples in that order
 * (counts[0] + counts[1] + counts[2] triples, at most max_units triples,
 * else FDTD_EINVAL).  The two adjoint lists together cover every unit of the
 * grid exactly once. */
int fdtd_reverse_units(int nx, int ny, int nz, int P, int zchunk, int* counts, int* units,
                       int max_units);

/* The deep units of the two-step forward (FDTD_OPT_FORWARD = 3) for an
 * nx x ny x nz grid with a P-cell CPML and split z chunks of zchunk planes:
 * box[0..5] = ix0, ix1, iy0, iy1, iz0, iz1, the tiles [ix0, ix1) x [iy0,
 * iy1) (x0 = 32 ix, y0 = 8 iy) and whole chunks [iz0, iz1) (planes [k0, k1))
 * for which the cells x in [x0 - 2, x0 + 34), y in [y0 - 2, y0 + 9), z in
 * [k0 - 2, k1] (where a two-step pass evaluates the intermediate level) all
 * lie in the interior [P, n - P) of every axis.  All zero when there are
 * none.  Host only; FDTD_EINVAL on NULL or non-positive sizes. */
int fdtd_deep_units(int nx, int ny, int nz, int P, int zchunk, int* box);

/* Self-test of the bounded device waits (failure detection without a
 * fault): one CTA arms an mbarrier for a copy that is never issued and waits
 * on it with the same bounded wait the TMA pipelines use, giving up after
 * limit_cycles (> 0) SM clock cycles.  On giving up it ORs the timeout bit
 * (4) into *d_flag (device, one unsigned, caller-owned and zeroed) and the
 * call returns FDTD_ETIMEOUT after synchronising the stream, with the CUDA
 * context still usable.  FDTD_EINVAL for a NULL flag or limit <= 0;
 * FDTD_ECUDA if the launch fails. */
int fdtd_selftest_wait(unsigned* d_flag, long long limit_cycles, void* cuda_stream);

/* The status a call returns for a device error word (host only, no device
 * use).  The kernels OR these bits into a word the host reads after each
 * run: 1 eps invalid (non-finite or < 1) -> FDTD_ENONFINITE; 4 a bounded
 * wait gave up -> FDTD_ETIMEOUT; 16 a bounds-checked store was dropped (the
 * checked test build) -> FDTD_ECUDA; 2 a non-finite gradient ->
 * FDTD_ENONFINITE; any other bit -> FDTD_ECUDA; 0 -> FDTD_OK.  With several
 * bits set the first in that order decides.  Every entry point that runs the
 * kernels (forward, backward, the group and no-allocation calls) maps the
 * word through this one rule. */
int fdtd_status_of_error_word(unsigned err_word);

/* ------------------------------------------------ no-allocation variant --- */

/* Largest workspace (bytes) fdtd_value_and_grad_noalloc can hold. */
#define FDTD_NOALLOC_SCRATCH_BYTES (64ull << 20)

/* Forward + backward without any device allocation, for callers that cannot
 * allocate device memory themselves: code that runs while someone else's
 * CUDA-graph capture is active (cudaMalloc is not permitted then), or
 * deployments whose device memory budget is fixed up front.  The paper has no
 * counterpart; this is a library convenience.
 *
 * Instead of a caller-bound workspace it uses one scratch array compiled into
 * the library: FDTD_NOALLOC_SCRATCH_BYTES (64 MiB) per GPU, reserved on every
 * GPU that loads the library and held until the process exits.  Problems
 * whose workspace (fdtd_workspace_bytes with the same rec) exceeds it are
 * rejected with FDTD_ENOMEM and a message giving both sizes.
 *
 * Arguments and results are those of fdtd_forward followed by fdtd_backward:
 * d_eps (device, float32 [nz][ny][nx]), seed, *objective (host), d_grad
 * (device, float32 design box).  Work is queued on the handle's stream and
 * the call blocks until done.  The first call on a device looks up the
 * scratch array's device address (cudaGetSymbolAddress) with that device
 * current, and the first call with a BDCT tape uploads the codec's basis
 * table (cudaMemcpyToSymbol, as any first BDCT use does); make those first
 * calls before any stream capture begins.  Device errors map to statuses as
 * in fdtd_status_of_error_word, after the forward and after the backward;
 * options are validated as for fdtd_forward (FDTD_EINVAL).  The call
 * itself calls no cudaMalloc / cudaFree, creates no stream, event or graph,
 * and clears every part of the scratch it reads before using it.  All calls
 * on a device share the one array, so calls that overlap on the GPU (from
 * several threads or streams) race: serialise them.  The handle's own
 * workspace binding, if any, is left untouched; after this call
 * fdtd_backward needs a new fdtd_forward. */
int fdtd_value_and_grad_noalloc(fdtd_handle* h, const float* d_eps, const fdtd_record_cfg* rec,
                                double seed, double* objective, float* d_grad);

#ifdef __cplusplus
}
#endif

#endif /* FDTD_GB300_H */
