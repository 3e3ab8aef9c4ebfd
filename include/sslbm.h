/*
 * sslbm.h -- C ABI of libsslbm.so, the GB300 (sm_103a) solver for the 2D SEIRD
 * reaction-diffusion model of De Rosis, "A distribution-free lattice Boltzmann
 * method for compartmental reaction-diffusion systems with application to epidemic
 * modelling" (arXiv 2603.19789).
 *
 * Two schemes advance the same problem:
 *   - the single-step simplified lattice Boltzmann method (SSLBM), Sec. II.C,
 *     Eq. (sslbm_final_clean) for S, E, I, R and the explicit update of Eq. (rhoD)
 *     for D -- the hot path;
 *   - the BGK lattice Boltzmann scheme of Sec. II.B, Eq. (pdf), on the D2Q5
 *     lattice with one population set per mobile compartment -- the comparison.
 *
 * Conventions shared by every entry point:
 *   - Every function returning int returns SSLBM_OK (0) or a negative status
 *     (SSLBM_ERR_*); sslbm_strerror() names it and sslbm_last_error() gives the
 *     detail of the last failure on the calling thread.  No function aborts the
 *     process or traps on the device.
 *   - Fields are 2D planes of ny rows by nx cells, row-major with x fastest
 *     (cell (x, y) at index y*nx + x), in the compartment order S, E, I, R, D
 *     (SSLBM_S .. SSLBM_D).  The paper's lattice is D2Q5 with dx in the lattice's
 *     length unit and dt in its time unit; densities are per cell.
 *   - Memory: the caller owns all device memory.  sslbm_workspace_bytes() says how
 *     much one solver needs; the caller allocates it (e.g. with PyTorch) and passes
 *     it to sslbm_create(); the library never allocates device memory.  The handle
 *     itself is a small host object owned by the library until sslbm_destroy().
 *   - Streams: all device work of a handle is ordered on the CUDA stream given at
 *     creation (or sslbm_set_stream()).  sslbm_step / bgk_step only enqueue work.
 *     Calls that return data to the host (sslbm_read to a host pointer,
 *     sslbm_diagnostics) synchronise that stream before returning.
 *   - A handle is not thread-safe: one thread drives it at a time.
 */
#ifndef SSLBM_H
#define SSLBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define SSLBM_OK 0
#define SSLBM_ERR_BAD_ARG (-1)     /* null pointer, bad enum, non-positive size ... */
#define SSLBM_ERR_UNSTABLE (-2)    /* parameters outside the scheme's stability range */
#define SSLBM_ERR_CUDA (-3)        /* a CUDA runtime call or kernel launch failed */
#define SSLBM_ERR_TIMEOUT (-4)     /* a bounded device wait ran out (ensemble barrier) */
#define SSLBM_ERR_NONFINITE (-5)   /* a diagnostic found NaN or Inf in the state */
#define SSLBM_ERR_WORKSPACE (-6)   /* workspace missing, too small or misaligned */
#define SSLBM_ERR_UNSUPPORTED (-7) /* valid request the library does not provide */
#define SSLBM_ERR_STATE (-8)       /* call out of order (e.g. stepping an unwritten scheme) */

/* ---- enumerations ------------------------------------------------------- */
enum { SSLBM_BC_PERIODIC = 0, SSLBM_BC_NOFLUX = 1 };
/* Storage and arithmetic precision of a solver's fields.
 *   FP64       : double fields, double arithmetic.
 *   FP32       : float fields, float arithmetic.
 *   FP32_DEV   : float fields; S is stored as its deviation sigma = s_ref - S from a
 *                uniform reference value, so that increments of order 1e-7 next to
 *                S ~ 1 are not rounded away.  Diffusion of sigma is that of S with the
 *                sign flipped (the stencil annihilates the constant s_ref exactly).
 *   FP32_KAHAN : float fields plus one float compensation plane per compartment;
 *                every step's increment is added with compensated (Kahan) summation.
 *   FP32_SPLIT : float fields; S is stored as a hi/lo pair -- its value plane v and a
 *                compensation plane c, S = v - c -- so that S keeps about twice FP32's
 *                precision at every value of S (the deviation storage keeps it only while
 *                S is near s_ref).  S's laplacian is taken in difference form on v minus
 *                that of c, and S's increment is added with Kahan summation; E, I, R, D
 *                are plain FP32.  Six planes: 48 bytes per cell-step.
 *   FP64_DW    : FP64-accurate fields in FP32 arithmetic: every value is a double word
 *                hi + lo of two floats (about 48 significant bits), stored as the Kahan
 *                storage's ten planes (hi, and the compensation -lo), and the update of
 *                FP64 is carried out in double-word arithmetic (the error-free building
 *                blocks of Joldes, Muller and Popescu, ACM TOMS 2017: relative error of
 *                order 2^-46 per operation), with the laplacian in difference form.  The
 *                exponent range is FP32's: values below 1e-38 lose precision, and an
 *                infection front whose leading edge lies below the smallest float (1.4e-45)
 *                in FP64 arrives shifted, as in every FP32 storage.  D2Q5 SSLBM, one step
 *                per launch; 80 bytes per cell-step. */
enum { SSLBM_FP64 = 0, SSLBM_FP32 = 1, SSLBM_FP32_DEV = 2, SSLBM_FP32_KAHAN = 3, SSLBM_FP32_SPLIT = 4,
       SSLBM_FP64_DW = 5 };
enum { SSLBM_SCHEME_SSLBM = 0, SSLBM_SCHEME_BGK = 1 };
enum { SSLBM_S = 0, SSLBM_E = 1, SSLBM_I = 2, SSLBM_R = 3, SSLBM_D = 4, SSLBM_NCOMP = 5 };
enum { SSLBM_ALL = -1 }; /* comp argument: all five planes, consecutive */
enum { SSLBM_DT_F64 = 0, SSLBM_DT_F32 = 1 };
/* schemes bitmask of sslbm_grid */
enum { SSLBM_WANT_SSLBM = 1, SSLBM_WANT_BGK = 2 };
/* lattice of sslbm_grid.  D2Q9 (Sec. II.C, isotropy discussion): rho_f and rho_b summed over
 * the nine velocities (weights 4/9, 1/9, 1/36), the isotropic 9-point Laplacian; stable for
 * 1/2 <= tau <= 13/8 (max(1 - Lambda9) = 8/9); no-flux walls as halfway bounce-back (a link
 * leaving the domain sees the cell's own value), which conserves the population exactly. */
enum { SSLBM_LATTICE_D2Q5 = 0, SSLBM_LATTICE_D2Q9 = 1, SSLBM_LATTICE_D2Q5_SLBM = 2, SSLBM_LATTICE_D2Q5_VARD = 3 };
/* SSLBM_LATTICE_D2Q5_SLBM: the two-pass simplified LBM of Eqs. (SLBM1, SLBM2) on D2Q5,
 * predictor rho* = sum_i w_i rho(x - c_i) and corrector
 * rho(t + dt) = rho* + (tau - 1)(sum_i w_i rho*(x + c_i) - rho) + Psi dt (two kernels per
 * step, four extra planes of workspace); stable for 1/2 <= tau <= 7/4; kept for comparison
 * with the single-step SSLBM, which needs one pass. */
/* SSLBM_LATTICE_D2Q5_VARD: the D2Q5 SSLBM with spatially varying, axis-anisotropic
 * diffusion, set per cell by sslbm_set_diffusivity_scale (Sec. IV lists this extension as
 * future work; the discretisation is this library's reading, given there). */

/* ---- problem description (Sec. II.A problem statement, Sec. III test case) -- */
typedef struct sslbm_grid {
  int64_t nx, ny;      /* lattice cells along x and y, each >= 1 */
  double dx, dt;       /* lattice spacing and time step (> 0); lattice units: 1, 1 */
  int32_t bc;          /* SSLBM_BC_PERIODIC or SSLBM_BC_NOFLUX (homogeneous Neumann,
                          cell-centred mirror; BGK: halfway bounce-back) */
  int32_t precision;   /* SSLBM_FP64 .. SSLBM_FP64_DW (BGK supports FP64 and FP32) */
  int32_t schemes;     /* SSLBM_WANT_SSLBM | SSLBM_WANT_BGK: which state to hold */
  int32_t lattice;     /* SSLBM_LATTICE_D2Q5 (0), SSLBM_LATTICE_D2Q9 (1),
                          SSLBM_LATTICE_D2Q5_SLBM (2) or SSLBM_LATTICE_D2Q5_VARD (3); 1 to 3:
                          SSLBM scheme only, FP64 or FP32; temporal blocking for FP32 on
                          D2Q9 and D2Q5_VARD (sslbm_set_blocking) */
} sslbm_grid;

/* Epidemiological parameters in the notation of Table I:
 * beta contact rate, alpha incubation rate (inverse mean incubation period),
 * gamma removal rate (I -> R or D), phi infection fatality ratio (0 <= phi <= 1).
 * Rates are per unit of dt.  Diffusion: either physical coefficients d[C]
 * (units dx^2 / dt, d[SSLBM_D] must be 0) converted with Eq. (diffusivity),
 * tau = 3 d dt / dx^2 + 1/2, or relaxation times tau[C] directly (use_tau != 0).
 * Stability (von Neumann analysis of Sec. II.C with the amplification
 * G = 1 - (2 tau - 1)(1 - Lambda)): 1/2 <= tau <= 5/4 for each mobile compartment
 * (13/8 on D2Q9, 7/4 for the two-pass SLBM), otherwise sslbm_create returns SSLBM_ERR_UNSTABLE.  With strict != 0
 * the nonnegativity condition 4 d_lattice + (outflow rate) dt <= 1 (20/6 d_lattice on
 * D2Q9; outflow beta for S, alpha for E, gamma for I) is enforced as well. */
typedef struct sslbm_params {
  double beta, alpha, gamma, phi;
  double d[5];        /* S, E, I, R, D */
  double tau[4];      /* S, E, I, R (read when use_tau != 0) */
  double s_ref;       /* FP32_DEV: reference value of S (typically the total density) */
  int32_t use_tau;
  int32_t strict;
} sslbm_params;

typedef struct sslbm_handle sslbm_handle;

/* ---- lifecycle -------------------------------------------------------------- */

/* Name of a status code (static string, never NULL). */
const char* sslbm_strerror(int status);

/* Detail of the last failure on the calling thread (static thread-local buffer). */
const char* sslbm_last_error(void);

/* Library version as major*10000 + minor*100 + patch. */
int sslbm_version(void);

/* Bytes of device workspace a solver for grid g needs (both ping-pong state
 * buffers of each requested scheme, the diagnostics scratch and padding).
 * Writes *bytes; returns SSLBM_ERR_BAD_ARG for an invalid grid. */
int sslbm_workspace_bytes(const sslbm_grid* g, size_t* bytes);

/* Create a solver.  g, p: problem (copied).  dev_ws: caller-owned device memory of
 * at least sslbm_workspace_bytes(g) bytes, 256-byte aligned, which must outlive the
 * handle.  stream: a cudaStream_t (NULL = legacy default stream).  On success
 * *out receives the handle and the state of each scheme is zero until written.
 * Validates the parameters (see sslbm_params) and converts d -> tau with
 * Eq. (diffusivity). */
int sslbm_create(const sslbm_grid* g, const sslbm_params* p, void* dev_ws, size_t ws_bytes,
                 void* stream, sslbm_handle** out);

/* Change the stream subsequent work is ordered on. */
int sslbm_set_stream(sslbm_handle* h, void* stream);

/* Destroy the handle (host object only; the caller frees the workspace afterwards,
 * once work on the stream has finished).  NULL is accepted. */
void sslbm_destroy(sslbm_handle* h);

/* ---- state transfer ------------------------------------------------------------ */

/* Set compartment comp (SSLBM_S..SSLBM_D, or SSLBM_ALL for five consecutive planes)
 * of scheme `scheme` from src: ny*nx values of type src_dtype (SSLBM_DT_F64 or
 * SSLBM_DT_F32) per plane, row-major, on the host (src_on_device = 0, pageable or
 * pinned) or the device (src_on_device = 1).  Values are rounded to the solver's
 * precision.  For BGK the populations of the written compartments are set to the
 * equilibrium f_i = w_i rho (Sec. II.B; the initial populations are not stated in
 * the paper).  FP32_KAHAN and FP64_DW keep the rounding residue of each written value in
 * its compensation plane, so FP64 input is represented to 2^-48 relative (within FP32's
 * exponent range).  When comp is SSLBM_ALL
 * the scheme's step counter is reset.  Host sources are consumed before the call returns. */
int sslbm_write(sslbm_handle* h, int scheme, int comp, const void* src, int src_dtype,
                int src_on_device);

/* Copy compartment comp (or SSLBM_ALL) of scheme `scheme` to dst in dst_dtype; for
 * BGK the density rho = sum_i f_i.  FP32_DEV returns S = s_ref - sigma, FP32_KAHAN the
 * compensated value and FP64_DW hi + lo, each evaluated in double precision.
 * A host destination synchronises the stream; a device destination is stream-ordered. */
int sslbm_read(sslbm_handle* h, int scheme, int comp, void* dst, int dst_dtype, int dst_on_device);

/* Per-cell diffusivity scale fields of a SSLBM_LATTICE_D2Q5_VARD solver: spatially varying
 * and axis-anisotropic diffusion, which Sec. IV lists as future work without a
 * discretisation.  The reading implemented here is the D2Q5 update in its link (flux) form:
 *   rho_new = rho_c + sum_i D_i (rho(x + c_i) - rho_c) + Psi dt,
 *   D_i = d_lattice^C (k_a(x) + k_a(x + c_i)) / 2,
 * with a = x on the two x links and a = y on the two y links, and
 * d_lattice^C = (tau^C - 1/2) / 3 from the params.  This is the conservative discretisation
 * of div(d(x) grad rho): both cells of a link share its coefficient, so the population is
 * conserved exactly (Sec. II.C).  Uniform fields of 1 give Eq. (sslbm_final_clean).  A link
 * through a no-flux wall carries nothing, and the periodic wrap links opposite edges.
 * kx, ky: ny*nx values each, row-major (x fastest), of type src_dtype (SSLBM_DT_F64 or
 * SSLBM_DT_F32), on the host (src_on_device = 0) or the device (1); ky == NULL uses kx for
 * both axes (isotropic).  Values are rounded to the solver's precision and copied into its
 * workspace; host sources are consumed before the call returns.
 * Validation, on the stored values: every value finite and >= 0, else SSLBM_ERR_BAD_ARG;
 * max_x sum_i D_i(x) <= 1 for every mobile compartment (links through a no-flux wall left
 * out), so that the centre weight of the update stays >= 0 and the diffusion part keeps a
 * maximum principle (with strict, the outflow rate times dt is added as in sslbm_params),
 * else SSLBM_ERR_UNSTABLE.  On any failure the solver has no fields until a call succeeds, and
 * sslbm_step returns SSLBM_ERR_BAD_ARG.  At create time a VARD solver only requires
 * tau >= 1/2; the fields decide stability.  Synchronises the stream.
 * Other lattices: SSLBM_ERR_UNSUPPORTED. */
int sslbm_set_diffusivity_scale(sslbm_handle* h, const void* kx, const void* ky, int src_dtype,
                                int src_on_device);

/* ---- time stepping ------------------------------------------------------------------ */

/* Advance the SSLBM state by n >= 0 time steps: Eq. (sslbm_final_clean) for S, E, I,
 * R with rho_f, rho_b, rho_c of Eqs. (rhof, rhob, rhoc) on the D2Q5 lattice and the
 * sources of Eq. (sources) at (x, t), and D(t+dt) = D + phi gamma I dt (Eq. rhoD).
 * On D2Q5 rho_f = rho_b, so the kernels evaluate the algebraically identical
 * rho_c + d_lattice (sum of the four neighbours - 4 rho_c) + Psi dt.
 * Several steps are fused per pass over memory (temporal blocking, depth set by
 * sslbm_set_blocking or sslbm_autotune; D2Q5 in every FP32 storage, D2Q9 and varying
 * diffusion in FP32); n steps
 * take ceil(n / depth) passes whose depths differ by at most one.  Results do not depend on
 * the depth: every depth performs the same floating-point operations in the same order.
 * Enqueues on the handle's stream and returns. */
int sslbm_step(sslbm_handle* h, int64_t n);

/* Advance the BGK state by n >= 0 steps of Eq. (pdf) (collide, then stream along
 * the D2Q5 links; no-flux walls by halfway bounce-back) with D by Eq. (rhoD). */
int bgk_step(sslbm_handle* h, int64_t n);

/* Steps taken by a scheme since its last full write. */
int64_t sslbm_steps_done(const sslbm_handle* h, int scheme);

/* ---- checkpoint / resume ------------------------------------------------------------- */

/* Not part of the paper's method (it has no restart); a facility of this library.
 * A checkpoint is the solver's state exactly as stored, so that a run resumed from it
 * gives the bits of the uninterrupted run.  sslbm_read / sslbm_write cannot do that for
 * every configuration: FP32_DEV returns S rebuilt from the stored deviation, FP32_KAHAN
 * the compensated value, FP64_DW hi + lo rounded to a double, and a BGK write sets
 * equilibrium populations.  Layout (a flat
 * byte buffer, host or device, owned by the caller): a 128-byte header (magic "SSLC",
 * version 2, nx, ny, precision, lattice, bc, schemes, the two step counters, the plane
 * counts, the element size and s_ref), then every stored plane in the solver's precision, each
 * ny*nx values row-major: the SSLBM planes (5; 6 for FP32_SPLIT; 10 with the Kahan
 * compensations or the double word's negated low parts) when
 * the handle holds that scheme, then the 21 BGK planes (20 populations, D) when it holds
 * BGK.  Parameters, blocking and the diffusivity scale fields are the handle's own and
 * are not part of a checkpoint. */

/* ---- debug build -------------------------------------------------------------------- */

/* Not part of the paper's method; a checking facility of this library.
 * Compiled with SSLBM_BOUNDS_CHECK (libsslbm_check.so, built by build.py --checked), the
 * hot-path kernels -- the fused pipeline tile of sslbm_step and the ensemble, the one-step
 * kernel, the BGK step and the diagnostics -- test the row and column indices of their
 * global loads and stores against the grid before each access, skip an access whose index
 * is out of range and record it.  sslbm_debug_bounds synchronises the current device,
 * returns the number of such indices since the last call, the first one, the limit it
 * missed and a site number (which check, offset by 100 per source file), then clears the
 * records.  count = 0 means every checked index was in range; value, limit and site are
 * then 0, 0 and -1.  Any pointer may be NULL.  sslbm_debug_bounds_probe checks value
 * against [0, limit) once on the device (site 999 + 300), with no memory access behind the
 * check: it exercises the recording path.  Release builds: both return
 * SSLBM_ERR_UNSUPPORTED. */
int sslbm_debug_bounds(long long* count, long long* value, long long* limit, int* site);
int sslbm_debug_bounds_probe(long long value, long long limit);

/* Bytes of a checkpoint of this handle. */
int sslbm_checkpoint_bytes(const sslbm_handle* h, size_t* bytes);

/* Copy the state and the step counters into dst (bytes >= sslbm_checkpoint_bytes, else
 * SSLBM_ERR_BAD_ARG), on the host (dst_on_device = 0) or the device (1).  Synchronises
 * the stream. */
int sslbm_checkpoint_save(sslbm_handle* h, void* dst, size_t bytes, int dst_on_device);

/* Restore state and step counters from a checkpoint made by a handle of the same grid
 * (nx, ny, precision, lattice, bc, schemes; under FP32_DEV also the same s_ref, since the
 * stored plane is the deviation s_ref - S).  A buffer that is too short, has another
 * magic or version, or was saved by a different configuration is rejected with
 * SSLBM_ERR_BAD_ARG before anything is copied.  A host source is consumed before the call
 * returns; a device source is read in stream order. */
int sslbm_checkpoint_load(sslbm_handle* h, const void* src, size_t bytes, int src_on_device);

/* ---- diagnostics (Sec. II.C 'Mass conservation') ------------------------------------ */

/* Per-compartment totals sum_x rho^C(x) accumulated in double precision, and the
 * peak infected density max_x I(x), of a scheme's current state.  totals: 5 doubles
 * (may be NULL), peak_I (may be NULL).  Synchronises the stream.  Returns
 * SSLBM_ERR_NONFINITE if any total is NaN or Inf (results still written). */
int sslbm_diagnostics(sslbm_handle* h, int scheme, double* totals, double* peak_I);

/* Fused diagnostics (on = 1; 0 turns them off, the default): the last pass of each
 * sslbm_step call also reduces its output to the totals and peak of sslbm_diagnostics,
 * so that a following sslbm_diagnostics(h, SSLBM_SCHEME_SSLBM, ...) reads them without a
 * pass over the state.  They are taken where that pass is temporally blocked on the D2Q5
 * lattice in SSLBM_FP32 or SSLBM_FP32_DEV and its grid has at most 1024 tiles (128-column
 * strips times row segments).  Any other step (also a call whose last pass is a single
 * step, as at depth 2 with an odd n), and any write or checkpoint load of the SSLBM state,
 * leaves sslbm_diagnostics to its own reduction.  The state written is the
 * same, and so are the results: each tile keeps FP32 TwoSum pairs of its output cells
 * (about twice FP32's precision per tile) and adds them in FP64 in a fixed order, so the
 * totals agree with the unfused reduction to rounding in FP64 and the peak exactly.
 * Returns SSLBM_ERR_BAD_ARG for a NULL handle or on not 0 or 1.  Not part of the paper. */
int sslbm_set_fused_diagnostics(sslbm_handle* h, int on);

/* Whether fused diagnostics are on (*on) and whether the last pass left those of the current
 * SSLBM state (*ready = 1: sslbm_diagnostics reads them without a pass over the state).
 * Either pointer may be NULL.  SSLBM_ERR_BAD_ARG for a NULL handle. */
int sslbm_get_fused_diagnostics(const sslbm_handle* h, int* on, int* ready);

/* Totals and peak infected of caller-provided fields, allocating no device memory.
 * The paper has no counterpart: this serves callers that hold device buffers but
 * cannot allocate -- e.g. a monitoring hook inside another framework's time loop whose
 * memory pool owns the free device memory (a cudaMalloc could fail, fragment the pool
 * or synchronise the device), or a plain C caller with no allocator for this device --
 * and so cannot give sslbm_create() the workspace sslbm_diagnostics() uses.
 * fields: device pointer to five planes S, E, I, R, D of ny x nx values each, laid out
 * [5][ny][nx] (the layout sslbm_read() returns), of type dtype (SSLBM_DT_F64 or
 * SSLBM_DT_F32).  totals (5 doubles) and peak_I are host outputs (either may be NULL).
 * stream: a cudaStream_t (NULL = legacy default stream); the call synchronises it.
 * Limit: ny <= 16384 rows (the scratch is a built-in 768 KiB device array, one slot
 * per row); larger ny returns SSLBM_ERR_BAD_ARG.  No cudaMalloc, cudaFree or
 * allocating library routine is called.  The array itself is device memory of the
 * library's image: CUDA reserves it when it loads this code on a device, which under
 * CUDA's default lazy module loading happens at the first call on that device -- so that
 * first call does claim 768 KiB in the caller's context.  A caller that must not see even
 * that make the first call at set-up, while allocation is still allowed, or runs with
 * CUDA_MODULE_LOADING=EAGER (the reservation then happens when the context is created).
 * The first call on each device also looks up the array's device address (with that
 * device current) and should come before any stream capture.  All calls on a device share the array and it keeps the last call's
 * partial sums; calls that overlap on the GPU race on it, so order them on one stream.
 * Returns SSLBM_ERR_NONFINITE if a total is NaN or Inf (results still written). */
int sslbm_diagnostics_noalloc(const void* fields, int dtype, int64_t nx, int64_t ny,
                              double* totals, double* peak_I, void* stream);

/* ---- tuning --------------------------------------------------------------------------- */

/* Temporal-blocking depth k (steps fused per pass, 1..SSLBM_MAX_DEPTH) and the
 * kernel's row-segment length seg_rows (0 = automatic).  k = 0 restores the default (4
 * where a blocked kernel exists, else 1).  The blocked kernels cover the D2Q5 lattice in
 * SSLBM_FP32, SSLBM_FP32_DEV, SSLBM_FP32_SPLIT and SSLBM_FP32_KAHAN, and the D2Q9 and
 * varying-diffusion lattices in SSLBM_FP32; k > 1 elsewhere returns SSLBM_ERR_UNSUPPORTED. */
#define SSLBM_MAX_DEPTH 8
int sslbm_set_blocking(sslbm_handle* h, int k, int seg_rows);

/* Autotuner: choose the blocking depth (1..SSLBM_MAX_DEPTH) and segment length for this
 * handle's grid, precision and lattice (D2Q5, D2Q9 or varying diffusion, whose scale fields
 * must be set; others: SSLBM_ERR_UNSUPPORTED) by
 * timing candidate launches on the handle's stream.  The candidates read the current state
 * and write the spare buffer, so the state is left unchanged.  budget_ms bounds the search
 * (0 = 300 ms).  The choice is cached per (device, nx, ny, precision, lattice, boundary)
 * for the life of the process, applied to the
 * handle, and returned through depth, seg_rows and ms_per_step (each may be NULL).
 * Synchronises the stream.  Not part of the paper (which gives no implementation). */
int sslbm_autotune(sslbm_handle* h, double budget_ms, int* depth, int* seg_rows,
                   double* ms_per_step);

/* Current blocking depth and segment length. */
int sslbm_get_blocking(const sslbm_handle* h, int* k, int* seg_rows);

/* ---- ensembles: many scenarios in one persistent launch ---------------------------------
 * Not in the paper (which runs one scenario at a time): a batch of independent SEIRD
 * scenarios, each on its own periodic grid (nx a multiple of 4) with its own rates and
 * diffusivities, all advanced by the SSLBM update of sslbm_step with one persistent,
 * CUDA-graph-captured launch per run.  The caller owns the device workspace. */
typedef struct sslbm_scenario {
  int64_t nx, ny;                  /* periodic grid of this scenario */
  double dx, dt;                   /* lattice spacing and time step (> 0) */
  double beta, alpha, gamma, phi;  /* Table I notation */
  double d[5];                     /* diffusivities S, E, I, R, D (d[D] = 0), Eq. (diffusivity) */
  double s_ref;                    /* FP32_DEV reference value of S */
} sslbm_scenario;

typedef struct sslbm_ensemble sslbm_ensemble;

/* Workspace bytes for n scenarios in the given precision (SSLBM_FP32, SSLBM_FP32_DEV or
 * SSLBM_FP32_SPLIT; the split storage keeps a sixth plane per scenario, the compensation of S;
 * others: SSLBM_ERR_UNSUPPORTED). */
int sslbm_ensemble_workspace_bytes(int n, const sslbm_scenario* sc, int precision, size_t* bytes);

/* Create an ensemble (scenarios copied; states zero until written).  dev_ws: caller-owned,
 * 256-byte aligned device memory of at least sslbm_ensemble_workspace_bytes bytes.
 * Returns SSLBM_ERR_UNSTABLE when a relaxation time exceeds 5/4. */
int sslbm_ensemble_create(int n, const sslbm_scenario* sc, int precision, void* dev_ws,
                          size_t ws_bytes, void* stream, sslbm_ensemble** out);

void sslbm_ensemble_destroy(sslbm_ensemble* e);

/* Tile shape of the persistent launch: steps fused per pass (depth in {2..6, 8}) and the
 * row-segment length of a tile (>= 4 * depth); the tile width is one 128-column strip. */
int sslbm_ensemble_set_tiling(sslbm_ensemble* e, int depth, int seg_rows);
int sslbm_ensemble_get_tiling(const sslbm_ensemble* e, int* depth, int* seg_rows);

/* Bound on each dependency wait of the persistent launch (polls, default 2^24), and a
 * fault-injection hook for tests: the work item numbered stall_item (-1 = none) never
 * reports completion, so the waits that depend on it run out and sslbm_ensemble_run
 * returns SSLBM_ERR_TIMEOUT instead of hanging.  After a timeout the states are undefined. */
int sslbm_ensemble_set_wait_limit(sslbm_ensemble* e, long long spin_limit, long long stall_item);

/* Set / get all five planes ([5][ny][nx]) of scenario idx, as in sslbm_write / sslbm_read
 * (FP64 or FP32 values; host or device memory; under FP32_SPLIT a write sets the compensation
 * of S to zero and a read returns value - compensation).  Both synchronise the stream. */
int sslbm_ensemble_write(sslbm_ensemble* e, int idx, const void* src, int src_dtype, int on_device);
int sslbm_ensemble_read(sslbm_ensemble* e, int idx, void* dst, int dst_dtype, int on_device);

/* Advance every scenario by nsteps SSLBM steps: nsteps / depth fused step-blocks in one
 * persistent launch (replayed from a cached CUDA graph), the remainder by one-step
 * launches.  Synchronises the stream to check the wait status (SSLBM_ERR_TIMEOUT). */
int sslbm_ensemble_run(sslbm_ensemble* e, int64_t nsteps);

/* Per-scenario totals (n x 5 doubles, row = scenario) and peaks of I (n doubles), as in
 * sslbm_diagnostics.  Either pointer may be NULL. */
int sslbm_ensemble_diagnostics(sslbm_ensemble* e, double* totals, double* peak_I);

/* Autotuner for the ensemble launch: times trial_blocks step-blocks (0 = 3) for each
 * depth in {2, 3, 4, 6, 8} and segment length in {32, 64, 128, 256}, keeps the fastest
 * per lattice step, and returns it (pointers may be NULL).  The trials run on the current
 * contents and the states are cleared to zero afterwards, so call it before writing the
 * initial states.  Synchronises the stream. */
int sslbm_ensemble_autotune(sslbm_ensemble* e, int trial_blocks, int* depth, int* seg_rows,
                            double* ms_per_step);

int64_t sslbm_ensemble_steps_done(const sslbm_ensemble* e);

/* Checkpoint / resume of an ensemble (not part of the paper's method), as sslbm_checkpoint_*
 * for one grid: the stored FP32
 * planes of every scenario (sigma = s_ref - S under FP32_DEV, the sixth plane under
 * FP32_SPLIT, as stored) and the step
 * counter, so that a resumed run gives the bits of the uninterrupted one.  Layout: a 64-byte
 * header (magic "SSLE", version 2, n, precision, steps), then (nx, ny, s_ref) of every
 * scenario as two int64 and a double, padded to a multiple of 128 bytes, then per scenario
 * its five planes of ny*nx floats, row-major.  Other scenario parameters and the tiling are
 * the handle's own and not saved.  A load checks magic, version, the scenario count, the
 * precision, every grid size and, under FP32_DEV, every s_ref before it copies anything
 * (SSLBM_ERR_BAD_ARG otherwise).  Save synchronises the stream; a load
 * from the host consumes its source before returning, one from the device is stream-ordered. */
int sslbm_ensemble_checkpoint_bytes(const sslbm_ensemble* e, size_t* bytes);
int sslbm_ensemble_checkpoint_save(sslbm_ensemble* e, void* dst, size_t bytes, int dst_on_device);
int sslbm_ensemble_checkpoint_load(sslbm_ensemble* e, const void* src, size_t bytes, int src_on_device);

/* ---- fourth-order finite-difference reference (Sec. III) ----------------------------------
 * The paper's accuracy reference: classical RK4 in time with the fourth-order centred
 * Laplacian L4 u = sum over axes (-u[-2] + 16 u[-1] - 30 u[0] + 16 u[+1] - u[+2]) / (12 dx^2),
 *   d/dt C = Psi^C + d^C L4 C (C = S, E, I, R),   d/dt D = phi gamma I,
 * Psi from Eq. (sources) at every stage.  Boundaries: periodic wrap, or no-flux as the even
 * reflection about the boundary face (u[-1] = u[0], u[-2] = u[1]).  g: nx, ny, dx, dt, bc,
 * precision SSLBM_FP64 or SSLBM_FP32 (schemes and lattice are ignored).  p: beta, alpha,
 * gamma, phi and the physical diffusivities d[] (use_tau must be 0, d[D] = 0); RK4
 * stability needs d dt / dx^2 <= 0.26 for every compartment (else SSLBM_ERR_UNSTABLE).
 * State: five contiguous planes [5][ny][nx] in the workspace (4 states: u, two stage
 * states, the slope sum), caller-owned like the solver's. */
typedef struct sslbm_fd4 sslbm_fd4;
int sslbm_fd4_workspace_bytes(const sslbm_grid* g, size_t* bytes);
int sslbm_fd4_create(const sslbm_grid* g, const sslbm_params* p, void* dev_ws, size_t ws_bytes,
                     void* stream, sslbm_fd4** out);
void sslbm_fd4_destroy(sslbm_fd4* f);
/* The whole state, [5][ny][nx] FP64 or FP32, host or device; host transfers synchronise. */
int sslbm_fd4_write(sslbm_fd4* f, const void* src, int src_dtype, int src_on_device);
int sslbm_fd4_read(sslbm_fd4* f, void* dst, int dst_dtype, int dst_on_device);
/* n RK4 steps of dt (four stage launches each), stream-ordered. */
int sslbm_fd4_step(sslbm_fd4* f, int64_t n);
int64_t sslbm_fd4_steps_done(const sslbm_fd4* f);
/* Order of the Laplacian: 4 (default, the reference) or 2, the second-order centred
 * Laplacian sum over axes (u[-1] - 2 u[0] + u[+1]) / dx^2 with the same RK4, sources and
 * ghost rule ("FDM 2nd" of the cost comparison, Table tab:timing). */
int sslbm_fd4_set_order(sslbm_fd4* f, int order);

/* ---- learned surrogate -------------------------------------------------------------------
 * Not in the paper.  A Fourier-neural-operator-style network that maps the five SEIRD
 * fields of a periodic n x n grid to the fields 20 SSLBM steps later.  With the infection
 * scale s = max over the grid of (E, I) (at least 1e-12), e = (log10 s + 4)/4 and
 * s' = 10^(4e - 4), the input has 8 channels
 *   x = [S, E/s', I/s', R, D, (R0 - 2.6)/1.4, log10(d) + 2, e]
 * and the network is
 *   h0 = A0 x + a0; z_l = K_l(h_{l-1}) + B_l h_{l-1} + b_l, h_l = gelu(z_l) (l < L), h_L = z_L;
 *   delta = Q2 gelu(Q1 h_L + q1) + q2;  v_c = sigma_c max(x_c + delta_c, 0),
 *   sigma = (1, s', s', 1, 1);  y = v (sum u / sum v) (0 if sum v = 0), u_c = sigma_c x_c,
 * sums over a sample, K_l a spectral convolution on the kx in {0..m-1, n-m..n-1},
 * ky in {0..m-1} Fourier modes with complex weights R_l[i][o][kx][ky].  E and I enter and
 * leave in units of the infection scale, so the early exponential phase is the same problem
 * at every amplitude; the clamp makes every density of y nonnegative and the rescale makes y
 * hold the total population of its input, by construction. 
 * Parameters are one flat FP32 vector in the order A0[W][8], a0[W],
 * {R_l[W][W][2m][m][2], B_l[W][W], b_l[W]}_{l=1..L}, Q1[H][W], q1[H], Q2[5][H], q2[5].
 * Dense contractions run on BF16 tensor cores with FP32 accumulation; activations are
 * BF16, parameters, gradients and Adam moments FP32.  For (W, m, H) = (32, 12, 64) or
 * (16, 8, 32) and n in {64, 128, 256} the forward pass runs as fused per-row kernels
 * (sslbm_fno_fused() says which); other shapes use one product per contraction.  All
 * tensors passed in are device pointers, FP32, laid out [batch][channel][n][n], 16-byte
 * aligned. */
typedef struct sslbm_fno_config {
  int32_t n;          /* grid side (periodic), 2 * modes <= n */
  int32_t width;      /* W: channels of the hidden layers (<= 64) */
  int32_t modes;      /* m: retained modes per direction (2m x m kept) */
  int32_t layers;     /* L: spectral layers (<= 16) */
  int32_t hidden;     /* H: width of the projection (<= 64) */
  int32_t max_batch;  /* largest batch a call may use (sizes the activations) */
} sslbm_fno_config;

typedef struct sslbm_fno sslbm_fno;

int sslbm_fno_workspace_bytes(const sslbm_fno_config* c, size_t* bytes);
int sslbm_fno_create(const sslbm_fno_config* c, void* dev_ws, size_t ws_bytes, void* stream,
                     sslbm_fno** out);
void sslbm_fno_destroy(sslbm_fno* f);
/* Number of parameters (-1 for a NULL handle). */
int64_t sslbm_fno_num_params(const sslbm_fno* f);
/* Set (also resets the Adam moments) / get the flat FP32 parameters, host or device memory. */
int sslbm_fno_set_params(sslbm_fno* f, const float* theta, int on_device);
int sslbm_fno_get_params(sslbm_fno* f, float* theta, int on_device);
/* Gradients of the last backward pass (flat, parameter order). */
int sslbm_fno_get_grads(sslbm_fno* f, float* grad, int on_device);
/* x[b] (8 channels, above) from states u[b][5][n][n] and per-scenario R0[b], log10(d)[b]. */
int sslbm_fno_make_input(sslbm_fno* f, int batch, const float* u, const float* r0,
                         const float* log10d, float* x);
/* y[b][5][n][n] = network(x[b]); keeps the activations for a following backward pass. */
int sslbm_fno_forward(sslbm_fno* f, int batch, const float* x, float* y);
/* The same y without keeping the activations (the rollout's call; a following backward
 * pass returns SSLBM_ERR_STATE). */
int sslbm_fno_infer(sslbm_fno* f, int batch, const float* x, float* y);
/* 1 when this configuration runs the fused forward kernels, 0 otherwise, < 0 on error. */
int sslbm_fno_fused(const sslbm_fno* f);
/* Parameter gradients of a scalar loss with dL/dy = dy, after sslbm_fno_forward on x with
 * the same batch (SSLBM_ERR_STATE otherwise). */
int sslbm_fno_backward(sslbm_fno* f, int batch, const float* x, const float* dy);
/* Adam hyper-parameters (defaults 0.9, 0.999, 1e-8, no weight decay). */
int sslbm_fno_set_adam(sslbm_fno* f, float beta1, float beta2, float eps, float weight_decay);
/* Weights (>= 0, default 0) of the two residual terms of the training loss:
 *   loss = mse_w + mass_weight mean_b r_b^2 + neg_weight mean_b n_b^2,
 *   mse_w = mean of ((y - t) / sigma_c)^2,  r_b = (sum y_b - sum t_b) / sum t_b,
 *   n_b = sum max(-y_b, 0) / sum t_b,
 * which teach the network to pass the conservation and nonnegativity checks of
 * sslbm_fno_check_project. */
int sslbm_fno_set_loss_weights(sslbm_fno* f, float mass_weight, float neg_weight);
/* Bound on each wait of the surrogate's tensor-core products for their MMAs (polls, default
 * 2^24; 0 restores it), and a fault-injection hook for tests: with stall != 0 the products
 * issue neither their MMAs nor the completion signal, so every wait runs out with no
 * tensor-core work in flight, the products write NaN and sslbm_fno_train_step returns
 * SSLBM_ERR_TIMEOUT instead of hanging.  The paper has no counterpart.  A product whose
 * wait runs out drains its MMAs (one more bounded wait) before it frees its tensor memory. */
int sslbm_fno_set_wait_limit(sslbm_fno* f, long long polls, int stall);
/* One training step on the loss of sslbm_fno_set_loss_weights: forward, loss, backward,
 * Adam with learning rate lr.  y_scratch and dy_scratch are [batch][5][n][n] device
 * buffers.  loss (host, may be NULL) receives mse_w before the update.  Synchronises the
 * stream; returns SSLBM_ERR_TIMEOUT if a tensor-core product of this step gave up waiting
 * for its MMAs (bounded wait; the product's tile is then NaN), in which case the Adam
 * update is skipped: parameters, moments and the step count stay as they were. */
int sslbm_fno_train_step(sslbm_fno* f, int batch, const float* x, const float* target,
                         float* y_scratch, float* dy_scratch, float lr, double* loss);
/* Residual checks of a prediction y against the input state u (both [batch][5][n][n]):
 * residuals[2b] = |sum y - sum u| / sum u (conservation of the total population),
 * residuals[2b+1] = sum max(-y, 0) / sum u (mass below zero).  Then y is projected in
 * place onto the admissible states:
 *   - with reach > 0, E, I, R and D are set to zero outside the domain of dependence of
 *     the input's infection: the cells farther than reach (periodic, per axis) from every
 *     cell where E + I or R + D exceeds 1e-6 of its maximum over the grid (reach = 20 for
 *     20 steps of the 5-point stencil, which moves information one cell per step);
 *   - every value is clamped at zero;
 *   - the state is rescaled to the input's total.
 * Synchronises the stream. */
int sslbm_fno_check_project(sslbm_fno* f, int batch, float* y, const float* u, int reach,
                            double* residuals);

/* ---- surrogate rollout with SSLBM fallback -------------------------------------------------
 * Not in the paper; the learned surrogate's serving loop (the learned-surrogate workload:
 * batched rollouts that fall back to the SSLBM when a conservation or nonnegativity residual
 * check fails).  Advances `batch` scenarios by `steps` surrogate steps of k_steps lattice
 * steps each (k_steps = the horizon the network was trained for, 20 for the surrogates this
 * library trains).  Each step: x = sslbm_fno_make_input(u), y = sslbm_fno_infer(x), then
 * the residuals of sslbm_fno_check_project (infinite for a non-finite prediction) and its
 * projection with `reach`; a scenario with conservation residual > mass_threshold or
 * negative mass > neg_threshold (either NaN also fails) takes the SSLBM instead: its state is
 * written into scenario b of `fallback`, the ensemble kernel advances it k_steps lattice
 * steps and the result replaces the prediction.  The rule of the learned-surrogate workload
 * is mass_threshold = 1e-4, neg_threshold = 0 (any negative density falls back).
 *   fallback: an ensemble whose scenarios 0..batch-1 are the rollout's scenarios (periodic
 *             n x n grids, their rates and diffusivities), FP32 or FP32_DEV; the rollout
 *             overwrites their states.  Its other scenarios are advanced too when it runs.
 *   u:        device, FP32 [batch][5][n][n]: the initial states in, the final states out.
 *   r0, log10d: device, FP32 [batch]: the network's per-scenario inputs.
 *   x_scratch, y_scratch: device, FP32 [batch][8][n][n] and [batch][5][n][n], 16-byte aligned.
 *   residuals: host [steps][batch][2] (conservation, negative mass) or NULL.
 *   fell_back: host [steps][batch], 1 where the SSLBM took the step, or NULL.
 *   stats:     host totals (or NULL).
 * Synchronises the surrogate's stream once per step (the residuals decide on the host) and
 * the ensemble's stream after each fallback; returns the first failing call's status. */
typedef struct sslbm_rollout_stats {
  int64_t surrogate_steps;       /* scenario-steps taken by the network */
  int64_t fallbacks;             /* scenario-steps taken by the SSLBM instead */
  int64_t failed_conservation;   /* scenario-steps whose conservation residual failed */
  int64_t failed_nonnegativity;  /* scenario-steps whose negative mass failed */
  double max_mass_residual;      /* largest finite conservation residual seen */
  double max_neg_residual;       /* largest finite negative-mass residual seen */
} sslbm_rollout_stats;

int sslbm_surrogate_rollout(sslbm_fno* f, sslbm_ensemble* fallback, int batch, int steps, int k_steps,
                            float* u, const float* r0, const float* log10d, float* x_scratch,
                            float* y_scratch, double mass_threshold, double neg_threshold, int reach,
                            double* residuals, unsigned char* fell_back, sslbm_rollout_stats* stats);

#ifdef __cplusplus
}
#endif
#endif /* SSLBM_H */
