/*
 * psatd.h -- C ABI of the GB300 (sm_103a) PSATD Maxwell step and its FDTD
 * comparators.
 *
 * Method (Blaclard, Vincenti, Lehe, Vay 2016, Sec. III.B item 2 and Table 1,
 * row "PSATD"): Maxwell's equations are solved in (k, t) space on a periodic
 * grid and integrated analytically over one time step, assuming the sources
 * J and rho are constant during the step; the scheme is dispersion-free and
 * has no Courant condition.  One step is: forward FFT of E, B, J (and rho),
 * the per-mode analytic push with C = cos(c|k|dt), S = sin(c|k|dt), inverse
 * FFT.  The FDTD comparators are the Yee and Cole-Karkkainen (CKC, beta = 1/4)
 * schemes of Sec. III.A / Table 1.
 *
 * PSATD-p (desc.order = p): on the staggered grid each component's spectrum
 * is first shifted to its true position (times exp(-i k_i d_i/2) per
 * staggered axis i), the update below is applied with k replaced by k_p,
 * k_p,i = (2/d_i) sum_{l=1}^{p/2} C_l sin((2l-1) k_i d_i/2) (C_l the staggered
 * Fornberg weights), and the spectra are shifted back; the Nyquist index keeps
 * k_i = +-pi/d_i there (the scheme propagates it).
 *
 * Per-mode update (c, eps0 explicit; kappa = k/|k|; x = c|k|dt):
 *   E' = C E + (1-C) kappa(kappa.E) + i c S kappa x B - S/(eps0 c k) J
 *        + (S/(c k) - dt)/eps0 kappa(kappa.J)                       [J-form]
 *   E' = C E + i c S kappa x B - S/(eps0 c k) J
 *        + i k/(eps0 k^2) [(S/x - 1) rho_np1 - (S/x - C) rho_n]      [rho-form]
 *   B' = C B + (1-C) kappa(kappa.B) - i S/(c k) k x E + i (1-C)/(eps0 c^2 k^2) k x J
 *   k = 0: E' = E - dt J/eps0, B' = B.
 * The Nyquist index of every even axis is treated as k_i = 0.
 *
 * Conventions common to every entry point
 *   - Arrays are caller-owned, one array per field component, x contiguous:
 *     2D [ny][nx], 3D [nz][ny][nx]; element type double for PSATD_FP64 and
 *     float for PSATD_FP32; base addresses 16-byte aligned.  Each array is
 *     memory of the plan's device (or managed memory), or pinned host memory
 *     (cudaHostAlloc / cudaHostRegister): the first and last passes then read
 *     and write the host arrays directly over the host-GPU link, with no
 *     separate copies.  Pageable host memory and other devices' memory are
 *     refused with PSATD_ERR_INVALID_ARG (cudaPointerGetAttributes, before
 *     any launch).
 *   - Staggering: PSATD is collocated (all components on the nodes); the FDTD
 *     arrays use the Yee positions Ex(i+1/2,j,k) Ey(i,j+1/2,k) Ez(i,j,k+1/2)
 *     Bx(i,j+1/2,k+1/2) By(i+1/2,j,k+1/2) Bz(i+1/2,j+1/2,k), J with E.
 *   - Time levels: E, B at t_n in, t_n+1 out (updated in place); J at
 *     t_n+1/2; rho_n at t_n, rho_np1 at t_n+1.  With nsteps > 1 the sources
 *     are held constant over the nsteps steps.
 *   - Every call is asynchronous and stream-ordered on the plan's CUDA stream
 *     (a cudaStream_t passed as void*; NULL = legacy default stream).  No call
 *     but psatd_plan_sync and psatd_kernel_times synchronises.
 *   - Host-side validation happens before any launch; an invalid argument
 *     returns PSATD_ERR_INVALID_ARG and launches nothing.  No exception crosses
 *     the ABI.  Message of the last failure: psatd_last_error(plan) (or
 *     psatd_last_error(NULL) for failures without a plan, thread-local).
 *   - A plan may be used by one host thread / one stream at a time.
 *   - Results are deterministic: no data-path atomics or reductions whose order
 *     varies, so a plan gives the same bits for the same inputs on every run,
 *     and changing lines per CTA (psatd_plan_set_launch cfg[0..4]) does not
 *     change them either; the radix schedule (cfg[5]) and the precision do.
 */
#ifndef PSATD_H
#define PSATD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PSATD_ABI_VERSION 1

typedef enum {
  PSATD_OK = 0,
  PSATD_ERR_INVALID_ARG = 1,  /* bad descriptor, null or misaligned pointer, bad count */
  PSATD_ERR_UNSUPPORTED = 2,  /* valid but not implemented (size, precision, layout)  */
  PSATD_ERR_OOM = 3,          /* device allocation failed                             */
  PSATD_ERR_CUDA = 4,         /* a CUDA runtime call or launch failed                 */
  PSATD_ERR_TIMEOUT = 5,      /* a bounded device-side wait expired                   */
  PSATD_ERR_NONFINITE = 6,    /* PSATD_FLAG_CHECKED: NaN or Inf in a step's output   */
  PSATD_ERR_BOUNDS = 7        /* PSATD_FLAG_CHECKED: a pass's index check failed      */
} psatd_status;

typedef enum {
  PSATD_FP64 = 0,        /* double storage and arithmetic                              */
  PSATD_FP32 = 1,        /* float storage; twiddles and C, S applied compensated (hi/lo) */
  PSATD_MIXED_BF16 = 2,  /* as PSATD_MIXED_FP16 with split-BF16 operands: a 8-bit
                            fixed-point head and two BF16 remainders, six products */
  PSATD_MIXED_FP16 = 3   /* float storage; every radix-16 FFT stage is a 16 x 16 DFT-
                            matrix contraction on the tensor cores (tcgen05) with
                            split-FP16 operands (hi + lo, per-row power-of-two scale,
                            three products) accumulated in FP32; the other stages,
                            twiddles and the push as PSATD_FP32.  PSATD step only. */
} psatd_precision;

typedef enum {
  PSATD_SRC_NONE = 0,    /* vacuum: J = rho = 0                     */
  PSATD_SRC_J = 1,       /* J-form: uses J                          */
  PSATD_SRC_J_RHO = 2    /* rho-form: uses J, rho_n and rho_np1     */
} psatd_source_form;

typedef enum {
  PSATD_FIELDS_3D6 = 0,   /* 3D, all six components                                 */
  PSATD_FIELDS_2D6 = 1,   /* 2D (x, y, uniform in z), all six components            */
  PSATD_FIELDS_2D_TE = 2, /* 2D: Ex, Ey, Bz (sources Jx, Jy, rho)                   */
  PSATD_FIELDS_2D_TM = 3  /* 2D: Ez, Bx, By (source Jz; no rho-form)                */
} psatd_layout;

typedef enum { PSATD_FDTD_YEE = 0, PSATD_FDTD_CKC = 1 } psatd_fdtd_scheme;

/* psatd_desc.flags bits.  PSATD_FLAG_AUTOTUNE: psatd_coeffs_init also picks
 * the launch shapes with the autotuner (psatd_plan_autotune with 5 timed
 * steps), or reuses the shapes found earlier in this process for the same
 * precision, layout, source form and sizes.  PSATD plans and batches only;
 * fdtd_step rejects it and psatd_step_noalloc ignores it. */
#define PSATD_FLAG_AUTOTUNE 1
/* PSATD_FLAG_PSTD: the plan's step is the pseudo-spectral time-domain scheme
 * (Table 1 row PSTD) instead of PSATD: the same transforms, and per mode the
 * leapfrog B -= (dt/2) i k x E; E += c^2 dt i k x B - dt J/eps0;
 * B -= (dt/2) i k x E (co-temporal E, B in and out, like fdtd_step).  Stable for
 * c dt |k| < 2 over the propagated modes (the caller's choice of dt); J-form or
 * vacuum only (INVALID_ARG with the rho-form); any order (k or k_p). */
#define PSATD_FLAG_PSTD 2
/* PSATD_FLAG_CHECKED: the checked mode.  (1) Index checks: before its first
 * access every CTA of every pass tests the element ranges it is about to read
 * and write (caller arrays, spectra, coefficient rows) against the extents the
 * plan knows; if any range falls outside, the CTA touches nothing and sets the
 * plan's device error word, and the next sync returns PSATD_ERR_BOUNDS (a bug
 * of this library, never of the caller's data).  (2) After every step the
 * output field arrays are scanned for NaN and Inf (one more read of the
 * outputs); a hit makes the next sync return PSATD_ERR_NONFINITE.  The sync
 * clears the word.  PSATD plans, batches and local decompositions;
 * psatd_step_noalloc and fdtd_step refuse it. */
#define PSATD_FLAG_CHECKED 4
/* PSATD_FLAG_TEST_STALL_MMA: a test hook of the failure path, for
 * PSATD_MIXED_FP16 / _BF16 plans only (INVALID_ARG otherwise).  The
 * tensor-core passes issue no MMA, so the first completion wait of every CTA
 * runs out after a short poll limit; the CTA then stops using the tensor
 * cores, frees its TMEM and finishes, and psatd_plan_sync returns
 * PSATD_ERR_TIMEOUT.  The step's output is not valid.  Never set it in
 * production use. */
#define PSATD_FLAG_TEST_STALL_MMA 8
/* PSATD_FLAG_TEST_SHORT_EXTENT: a test hook of the checked mode (with
 * PSATD_FLAG_CHECKED only, INVALID_ARG otherwise): every pass is told that each
 * array it touches is one element shorter than it is, so the index checks of
 * the CTAs reaching the last element fail, those CTAs skip their accesses and
 * psatd_plan_sync returns PSATD_ERR_BOUNDS.  The step's output is not valid. */
#define PSATD_FLAG_TEST_SHORT_EXTENT 16

/* Problem statement (the paper's arguments: grid sizes, cell sizes, dt, c, eps0). */
typedef struct {
  int32_t ndim;      /* 2 or 3 (must agree with layout)                           */
  int32_t layout;    /* psatd_layout                                              */
  int64_t n[3];      /* cells along x, y, z; n[2] = 1 in 2D                       */
  double d[3];       /* cell sizes dx, dy, dz (> 0; d[2] ignored in 2D)           */
  double dt;         /* time step (> 0; PSATD has no Courant limit)               */
  double c;          /* speed of light (> 0)                                      */
  double eps0;       /* vacuum permittivity (> 0)                                 */
  int32_t prec;      /* psatd_precision                                           */
  int32_t src;       /* psatd_source_form                                         */
  int32_t flags;     /* PSATD_FLAG_* bits (0: none)                               */
  int32_t order;     /* 0: all components on the nodes, exact wavenumbers k;
                        p (even, 2..256): PSATD-p (Table 1) on the staggered
                        (Yee) grid - components at the FDTD positions listed
                        above, k replaced by the order-p staggered-stencil
                        wavenumbers k_p (PSATD step only)                        */
} psatd_desc;

/* Field arrays, updated in place.  Entries of components absent from the
 * layout must be NULL (TE: E[0], E[1], B[2]; TM: E[2], B[0], B[1]).        */
typedef struct { void* E[3]; void* B[3]; } psatd_fields;

/* Source arrays, read only.  J entries of absent components must be NULL;
 * rho_n / rho_np1 are used by PSATD_SRC_J_RHO only.                        */
typedef struct { const void* J[3]; const void* rho_n; const void* rho_np1; } psatd_sources;

typedef struct psatd_plan_s* psatd_plan;

/* ABI version of the loaded library (PSATD_ABI_VERSION of its build). */
int32_t psatd_abi_version(void);

/* Create a PSATD plan for `desc` on `cuda_stream`.
 * Supported sizes: every n[i] a power of two, 16 <= n[0] <= 4096,
 * 8 <= n[1], n[2] <= 4096; with PSATD_FP32 also the mixed-radix lengths
 * n[0] = 6 * 2^k in [96, 3072] (x rows of n[0]/2 = 3 * 2^(k-1) points) and
 * n[1], n[2] = 3 * 2^k in [48, 3072] (radix-3 first stage), and
 * n[0] = 10 * 2^k in [160, 2560], n[1], n[2] = 5 * 2^k in [80, 1280] (radix-5
 * first stage), on any axis and combined freely with powers of two;
 * PSATD_FP64, PSATD_FP32,
 * PSATD_MIXED_FP16 or _BF16; flags from PSATD_FLAG_*.  A last axis of n
 * points needs (n_in + 1) * n * 8 (FP32) or 16 (FP64) bytes of shared memory
 * per CTA (UNSUPPORTED beyond the device's opt-in limit).
 * The mixed precisions also need n[0] >= 32, n[1], n[2] >= 16 and
 * at least 128 threads per CTA in every pass (n[0]/32 * min(32, n[1]) >= 128
 * for the x pass; UNSUPPORTED otherwise).
 * Owns: its spectral scratch (about n_in * (n0/2+1) * n1 * n2 complex values,
 * twice that in 3D), the twiddle tables and the k-space coefficient table,
 * allocated with cudaMalloc on the current device.  *out is set to NULL on
 * failure.  Errors: INVALID_ARG, UNSUPPORTED, OOM, CUDA.                   */
psatd_status psatd_plan_create(const psatd_desc* desc, void* cuda_stream, psatd_plan* out);

/* Fill the plan's tables on the device (FP64 arithmetic, rounded once to the
 * step precision; FP32 keeps hi/lo pairs of the twiddles and of C and S/|k|):
 * twiddles exp(-2 pi i j / n) per axis and, per |k|-octant entry,
 * C, S/|m|, (1-C)/|m|^2, (S/(ck)-dt)/(eps0 |m|^2), (S/x-1)/(eps0 g |m|^2),
 * (S/x-C)/(eps0 g |m|^2) with their k -> 0 limits, all scaled by 1/N.
 * Must be called once before psatd_step (psatd_step fails otherwise).
 * With PSATD_FLAG_AUTOTUNE it then runs (or recalls) the autotuner and is
 * synchronous.                                                              */
psatd_status psatd_coeffs_init(psatd_plan plan);

/* Autotuner (no counterpart in the paper; the launch shapes of the passes).
 * Times every valid candidate of each knob with CUDA events on the plan's
 * stream over `reps` steps (1..1000) of zero-filled scratch fields it
 * allocates and frees, keeps the fastest, and caches it for the process:
 *   lines per CTA of each transposing pass (x forward/inverse, y in 3D), and
 *   the fused pass's radix schedule (radix-8 or radix-16 stages, i.e. 8 or 16
 *   elements per thread; radix 16 only for the mixed precisions; for 3 * 2^k
 *   lengths only 12 elements per thread: a radix-12 first stage, then radix
 *   2 and 4) with its lines per CTA and component groups (below).
 * Results do not depend on the choice (same arithmetic, same order per line).
 * `report` (may be NULL) receives a one-line summary of the times, the chosen
 * ones marked '*', truncated to report_len - 1 bytes.  Synchronous.
 * Errors: INVALID_ARG (NULL plan, tables not initialised, reps out of range),
 * OOM (scratch), UNSUPPORTED, CUDA.                                         */
psatd_status psatd_plan_autotune(psatd_plan plan, int32_t reps, char* report, size_t report_len);

/* Launch shapes of the plan, as int32_t cfg[6]:
 *   cfg[0..3] log2(lines per CTA) of the x forward, y forward (3D), y inverse
 *             (3D) and x inverse passes (-1 / unused: 2D y passes);
 *   cfg[4]    lines per CTA of the fused pass;
 *   cfg[5]    its elements per thread: 8 (radix-8 stages), 16 (radix-16) or,
 *             for a last axis of 3 * 2^k points, 12 (radix 12, then 2/4).
 * psatd_plan_get_launch reports the shapes the next step will use.
 * psatd_plan_set_launch sets them (-1 entries: the built-in choice) after
 * checking each against the shapes the autotuner would consider
 * (INVALID_ARG otherwise); it rebuilds the fused axis's twiddle table when
 * cfg[5] changes, so it needs psatd_coeffs_init first.                    */
psatd_status psatd_plan_set_launch(psatd_plan plan, const int32_t cfg[6]);
psatd_status psatd_plan_get_launch(psatd_plan plan, int32_t cfg[6]);

/* Component groups of the fused pass (a launch shape, like cfg[4]): with G > 1
 * each line gets G thread groups that forward- and inverse-transform its
 * components in turn (group j: components j, j + G, ...; their own exchange
 * buffer and barrier each), meeting for the per-mode push; shared memory per
 * line grows from (n_in + 1) to (n_in + G) line buffers.  G = 1 is the plain
 * pass.  Tensor-core plans (PSATD_MIXED_*): 2 only, two 128-row groups that
 * transform component pairs in lockstep and share every tensor-core round
 * (measured slower than one group on GB300; kept as a launch shape).
 * Valid otherwise: 1 always; 2 or 4 for PSATD_FP32 plans whose fused-axis lines
 * have a multiple of 32 threads (length / elements per thread), at most 512
 * threads and 15 groups per CTA, an even number of modes per thread, and the
 * shared memory within the device's limit.  -1: the built-in choice, 2 where
 * lines have at least 64 threads and the one-group pass keeps fewer than 12
 * warps per SM resident (shared memory: many components on long lines, e.g.
 * 1024-point 3D rho-form lines), else 1.  Results
 * are bitwise the same for every G (each transform and each mode's update
 * runs the same arithmetic).  set: INVALID_ARG when the shape is not valid
 * for the plan's current lines per CTA and elements per thread (a later
 * psatd_plan_set_launch that makes it invalid falls back to 1).  get: the G
 * the next step uses.                                                     */
psatd_status psatd_plan_set_push_groups(psatd_plan plan, int32_t groups);
psatd_status psatd_plan_get_push_groups(psatd_plan plan, int32_t* groups);

/* Advance E, B by nsteps PSATD steps (nsteps >= 1).  `sources` may be NULL
 * for PSATD_SRC_NONE and must not be NULL otherwise.  Per step: forward
 * R2C/C2C FFT passes of every input component, the fused per-mode push with
 * the first inverse pass, the remaining inverse passes (C2R last).  Never
 * synchronises.  Errors: INVALID_ARG (missing/extra/misaligned pointer,
 * nsteps < 1, coefficients not initialised), CUDA.                          */
psatd_status psatd_step(psatd_plan plan, const psatd_fields* fields,
                        const psatd_sources* sources, int32_t nsteps);

/* Synchronise the plan's stream and report any asynchronous CUDA error, or
 * PSATD_ERR_BOUNDS when a checked plan's index check failed, or
 * PSATD_ERR_TIMEOUT when a bounded device-side wait gave up since the last
 * sync: the fused pass's wait for its bulk-copied inputs, or a tensor-core
 * pass's (PSATD_MIXED_FP16 / _BF16) wait for its MMAs (the CTA then skipped its
 * remaining tensor-core stages and freed its TMEM; the step's output is not
 * valid), or PSATD_ERR_NONFINITE when a checked plan (PSATD_FLAG_CHECKED)
 * saw NaN or Inf in a step's output since the last sync; the word is cleared. */
psatd_status psatd_plan_sync(psatd_plan plan);

/* Release the plan and everything it owns (synchronises its stream first).
 * NULL is accepted and ignored. */
psatd_status psatd_plan_destroy(psatd_plan plan);

/* Bytes of device memory the plan owns. */
size_t psatd_plan_workspace_bytes(psatd_plan plan);

/* Per-kernel CUDA-event timing of the plan's launches.  enable != 0 starts
 * recording an event pair around every launch on the plan's stream (and
 * clears earlier records).  psatd_kernel_times synchronises, then writes for
 * each kernel slot i < n_slots: its name (names[i] points into the library,
 * valid while the plan lives), the number of launches and the summed
 * milliseconds, and returns the number of slots used.                       */
psatd_status psatd_plan_set_timing(psatd_plan plan, int32_t enable);
int32_t psatd_kernel_times(psatd_plan plan, int32_t n_slots, const char** names,
                           int64_t* launches, double* total_ms);

/* Advance co-temporal E, B (Yee staggering) by nsteps FDTD steps:
 * B -= (dt/2) curl E;  E += dt (c^2 curl B - J/eps0);  B -= (dt/2) curl E.
 * scheme: PSATD_FDTD_YEE (2D or 3D) or PSATD_FDTD_CKC (2D only; the Faraday
 * differences are weighted 1-beta on the centre row and beta/2 on the two
 * transverse neighbour rows, beta = 1/4).  desc->src must be PSATD_SRC_NONE
 * or PSATD_SRC_J.  Sizes: any n[i] >= 2.  Launches on `cuda_stream`, no
 * allocation, no synchronisation.  Errors: INVALID_ARG, UNSUPPORTED, CUDA. */
psatd_status fdtd_step(const psatd_desc* desc, int32_t scheme, const psatd_fields* fields,
                       const psatd_sources* sources, int32_t nsteps, void* cuda_stream);

/* ---- batches of 2D patches --------------------------------------------
 * The paper advances many subdomains, each with its own local FFT
 * (Sec. II.A.3).  A batch holds npatch independent periodic 2D patches sharing
 * the base descriptor's layout (2D6, TE or TM), precision, source form, cell
 * sizes, dt, c and eps0; patch i has n[2i] x n[2i+1] cells (sizes as for
 * psatd_plan_create: powers of two, or 3 * 2^k lengths in FP32).  Fields and
 * sources of all patches are packed per component: one array per component
 * holding patch 0, patch 1, ... back to back (patch i at element offset
 * sum_{j<i} n[2j] n[2j+1]).
 * Patches of equal size form a class (own spectra and tables).  A step runs
 * the persistent passes below where the sizes allow; else one launch per pass
 * and class, forked from the batch's stream into up to four internal streams
 * that run the classes side by side, and joined back.  A call with nsteps > 1 on a
 * non-default stream records one step of all classes into a CUDA graph
 * (re-recorded when the field/source pointers change) and replays it nsteps
 * times.  Guard cells are part of each patch
 * (the caller fills them; no exchange between patches is done here).      */
typedef struct psatd_batch_s* psatd_batch;

/* Create a batch (allocates each class's spectra, tables and offset table
 * and fills the tables; synchronous).  *out = NULL on failure.
 * Errors: INVALID_ARG, UNSUPPORTED, OOM, CUDA (message: psatd_last_error(NULL)). */
psatd_status psatd_batch_create(const psatd_desc* base, int32_t npatch, const int64_t* n,
                                void* cuda_stream, psatd_batch* out);

/* Advance every patch by nsteps PSATD steps (sources held constant), as
 * psatd_step does for one grid.  Asynchronous. */
psatd_status psatd_batch_step(psatd_batch batch, const psatd_fields* fields,
                              const psatd_sources* sources, int32_t nsteps);

/* Total cells of the batch (sum over patches). */
int64_t psatd_batch_cells(psatd_batch batch);

/* Synchronise the batch's stream and report, as psatd_plan_sync does for each
 * size class, an asynchronous CUDA error, PSATD_ERR_TIMEOUT (tensor-core waits)
 * or PSATD_ERR_NONFINITE (PSATD_FLAG_CHECKED) since the last sync. */
psatd_status psatd_batch_sync(psatd_batch batch);

/* Persistent passes (selectable; per-class launches are the default).  When
 * every patch's line lengths allow it (FP32 or a mixed precision; x lines
 * n[2i]/2 of 32..512 points, or 48..384 = 3 * 2^k in FP32; last-axis lines
 * n[2i+1] of 64..1024, or 48..768 = 3 * 2^k in FP32), psatd_batch_set_persistent
 * (batch, 1) makes a step one launch per pass type (x forward, fused y pass, x
 * inverse) and per length family (powers of two, 3 * 2^k): the CTAs of each
 * launch stay resident and take the work of every patch from a device queue (an
 * atomic counter; the last CTA to finish resets it), so the passes run in stream
 * order with no wait inside a kernel.  psatd_batch_set_persistent(batch, 0)
 * returns to one launch per pass and size class on the branch streams described
 * above, which keeps a class's spectra in L2 between its passes and measured
 * faster; UNSUPPORTED when the sizes do not allow the persistent passes.  The
 * results are the same bits either way.  psatd_batch_launches_per_step: kernel launches of
 * one step in the current mode (without PSATD_FLAG_CHECKED's scans).  The
 * first step after the field or source pointers change uploads the classes'
 * argument tables (a synchronising copy, outside any graph capture). */
psatd_status psatd_batch_set_persistent(psatd_batch batch, int32_t enable);
int32_t psatd_batch_launches_per_step(psatd_batch batch);

/* Per-class launches on the branch streams (forked != 0, the default) or all on
 * the batch's own stream one class after another (forked = 0: no kernel of one
 * class overlaps another's, so per-launch event times are the kernels' own).
 * Synchronises the batch's streams; the same bits either way. */
psatd_status psatd_batch_set_branches(psatd_batch batch, int32_t forked);

/* Component groups of every size class's fused pass (psatd_plan_set_push_groups):
 * each class takes `groups` (2 or 4) where its shape admits them and one group
 * otherwise; 1 everywhere; -1 the built-in choice.  The per-class launches use
 * it (the persistent passes keep one group).  Synchronises the batch's streams;
 * the same bits either way.  INVALID_ARG for other values. */
psatd_status psatd_batch_set_push_groups(psatd_batch batch, int32_t groups);

/* Per-kernel CUDA-event timing of the batch, as psatd_plan_set_timing /
 * psatd_kernel_times do for a plan, summed over the size classes: enable != 0
 * records an event pair around every launch of every class (the recorded step
 * graph is recorded again with them, so each replay updates the pairs: after
 * a multi-step call they hold the last step's times).  psatd_batch_kernel_times
 * synchronises and writes per kernel slot its name, launches and summed ms.
 * Kernels of different classes may run at the same time on the batch's branch
 * streams, so a slot's summed time can exceed the step's wall time. */
psatd_status psatd_batch_set_timing(psatd_batch batch, int32_t enable);
int32_t psatd_batch_kernel_times(psatd_batch batch, int32_t n_slots, const char** names,
                                 int64_t* launches, double* total_ms);

/* Release the batch (synchronises its stream).  NULL is accepted. */
psatd_status psatd_batch_destroy(psatd_batch batch);

/* Local-FFT decomposition of one periodic 2D grid (Sec. II.A.3): the grid of
 * global->n[0] x global->n[1] cells is split into px x py patches of
 * ix = n[0]/px by iy = n[1]/py interior cells; every patch is extended by
 * `guard` cells on each side, which hold copies of the neighbouring cells
 * (periodic wrap at the grid's edges) refreshed before every step; each
 * extended patch is advanced by one PSATD step as a periodic domain of its own
 * (its own FFTs, all patches batched in one launch per pass), and the interiors
 * are written back.  The result differs from the global step by the truncation
 * error of the local transforms, which falls with the guard width.
 * global: layout 2D6, TE or TM; precision, source form, cell sizes, dt, c and
 * eps0 as in psatd_plan_create; n[0], n[1] need not be powers of two, but the
 * extended sizes ix + 2 guard and iy + 2 guard must satisfy psatd_plan_create's
 * limits.  Owns a plan of the extended size (px*py patches) and the packed
 * patch arrays (n_in * px*py * (ix+2g) * (iy+2g) values).
 * Errors: INVALID_ARG (NULL, px/py not dividing the grid, guard < 0),
 * UNSUPPORTED (3D, extended sizes out of range), OOM, CUDA.                 */
typedef struct psatd_local_s* psatd_local;
psatd_status psatd_local_create(const psatd_desc* global, int32_t px, int32_t py, int32_t guard,
                                void* cuda_stream, psatd_local* out);

/* Advance the global fields by nsteps local-FFT steps (sources held constant;
 * arrays as for psatd_step, of the global size).  Per step: guard refresh of
 * the fields (sources once per call), the batched patch step, write-back of the
 * interiors.  Asynchronous.  Errors as psatd_step.                           */
psatd_status psatd_local_step(psatd_local local, const psatd_fields* fields,
                              const psatd_sources* sources, int32_t nsteps);

/* The plan of the extended patches (timing, autotuning, launch shapes). */
psatd_plan psatd_local_plan(psatd_local local);

/* Release the decomposition (synchronises its stream).  NULL is accepted. */
psatd_status psatd_local_destroy(psatd_local local);

/* PSATD step without any device allocation, for callers that cannot call
 * cudaMalloc (e.g. code running where a foreign allocator owns all device
 * memory, or a host that must not allocate after start-up).  The paper has no
 * counterpart: this is a deployment variant of psatd_plan_create +
 * psatd_coeffs_init + psatd_step + psatd_plan_destroy in one call.
 *   Scratch: one fixed 16 MiB (16,777,216-byte) device array inside the
 *   library, held by every GPU that loads the library until the process exits.
 *   A call needs, each part rounded up to 256 bytes: the spectra
 *   n_in * (n0/2+1) * n1 * n2 complex values (twice that in 3D; 8 B each in
 *   FP32, 16 B in FP64), twiddles of 16 B per point of every axis, and the
 *   coefficient table (n0/2+1)(n1/2+1)(n2/2+1 in 3D) entries of 32 B (FP32) or
 *   64 B (FP64).  Larger grids are rejected with PSATD_ERR_UNSUPPORTED and a
 *   message naming the size: for FP32 2D TE J-form (n_in = 5) 768^2 fits and
 *   1024^2 does not.  The caller still passes (and owns) every field and source
 *   array.
 *   Set-up: the first call on a device looks up the array's device address
 *   (with that device current), and looks it up again when the device's context
 *   has changed since (after a device reset); make the first call, and the first
 *   call after a reset, before any stream capture.
 *   Each call rebuilds the twiddle and coefficient tables in the array (the
 *   array keeps the previous call's contents; the spectra are overwritten
 *   before they are read, so nothing needs clearing).
 *   All calls share the one array: calls whose work overlaps on the GPU (other
 *   streams, other host threads) race and corrupt each other's results.
 * Precision: PSATD_FP32 or PSATD_FP64 (others: PSATD_ERR_UNSUPPORTED).
 * Arguments and errors as psatd_plan_create and psatd_step; asynchronous.   */
psatd_status psatd_step_noalloc(const psatd_desc* desc, const psatd_fields* fields,
                                const psatd_sources* sources, int32_t nsteps, void* cuda_stream);

/* Fraunhofer far-field transform of a 2D field snapshot: the diagnostic of the
 * angularly resolved harmonic spectrum (Sec. II.B applies the Fraunhofer
 * diffraction integral to the reflected field of the simulation).  For every
 * wavevector k_j = (k[2j], k[2j+1]):
 *   U_j = sum_{x0 <= i < x1, y0 <= j' < y1} w_i v_j' F[j'][i]
 *         exp(-i (k[2j] i dx + k[2j+1] j' dy)) dx dy,
 * the far-field amplitude radiated towards direction k_j/|k_j| at wavenumber
 * |k_j| (harmonic n of a fundamental k0: the ring |k| = n k0).  w, v: Hann
 * apodisation sin^2(pi (i - x0 + 1/2)/(x1 - x0)) along x (apodise >= 1) and
 * along y (apodise == 2), else 1.
 * grid: ndim 2, n[0] = nx, n[1] = ny (the field's row length and rows), d[0],
 * d[1]; prec PSATD_FP32 (float field) or PSATD_FP64 (double); the other
 * members are ignored.  field: [ny][nx], x contiguous; window = {x0, x1, y0,
 * y1} (cells, half-open, inside the grid; rows of at most 8192 cells); k: nk
 * (kx, ky) pairs of doubles; out: nk (re, im) pairs of doubles, written.  The
 * field, k and out are device memory or pinned host memory of the current
 * device, caller-owned.  One launch on `cuda_stream`, no allocation, no
 * synchronisation; the sums are taken in a fixed order (deterministic), rows in
 * the field's precision, the phases and the sum over rows in FP64.
 * Errors: INVALID_ARG (NULL, empty or out-of-grid window, nk < 1, bad apodise,
 * inaccessible or misaligned pointer), UNSUPPORTED (3D, longer rows), CUDA.  */
psatd_status psatd_farfield(const psatd_desc* grid, const void* field, const int64_t window[4],
                            int32_t apodise, int32_t nk, const double* k, double* out,
                            void* cuda_stream);

/* Message of the last failure on `plan`, or of this thread's last failure
 * without a plan when plan == NULL.  Never NULL. */
const char* psatd_last_error(psatd_plan plan);

#ifdef __cplusplus
}
#endif

#endif /* PSATD_H */
