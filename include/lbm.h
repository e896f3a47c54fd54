/*
 * lbm.h -- C ABI of the GB300 (sm_103a) D2Q9 improved-MRT pseudopotential lattice
 * Boltzmann library, after Li, Luo & Li, "Lattice Boltzmann modeling of multiphase flows
 * at large density ratio with an improved pseudopotential model" (arXiv:1211.6932).
 *
 * Conventions shared by every entry point
 * ----------------------------------------
 *  - Return value: LBM_OK (0) on success, a negative LBM_E* code otherwise.  The message
 *    of the last failure is available from lbm_last_error(handle) (or
 *    lbm_last_error(NULL) for failures before a handle exists, kept per thread).
 *  - Lattice units: c = delta_t = 1, c_s^2 = 1/3.
 *  - Host field arrays are row-major (ny, nx) doubles: element (y, x) at y*nx + x.
 *    Host population arrays are (9, ny, nx) doubles: f_q(x, y) at q*nx*ny + y*nx + x, with
 *    the D2Q9 velocities in this order: e0 = (0,0), e1 = (1,0), e2 = (0,1), e3 = (-1,0),
 *    e4 = (0,-1), e5 = (1,1), e6 = (-1,1), e7 = (-1,-1), e8 = (1,-1).
 *    Populations are those at the current time before collision (the f of Eq. 1).
 *  - The library owns every device buffer of a handle; the caller owns every host buffer
 *    and every device buffer it passes in.  Pointers are only read during the call.
 *  - Work is queued on the handle's CUDA stream.  Calls that return data to the host
 *    synchronise that stream; lbm_step does not.
 *  - A handle is not thread-safe: one thread at a time.
 *  - Nothing here falls back to the CPU: without a usable CUDA device lbm_create returns
 *    LBM_ECUDA.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_OK 0
#define LBM_EINVAL (-1)    /* an argument is out of range; nothing was changed */
#define LBM_ENOMEM (-2)    /* a device or host allocation failed */
#define LBM_ECUDA (-3)     /* a CUDA runtime call failed (message names it) */
#define LBM_EUNSTABLE (-4) /* a density became non-finite or non-positive */
#define LBM_ETIMEOUT (-5)  /* a bounded device-side wait ran out (the kernel gave up and
                              returned; the state was not advanced correctly) */
#define LBM_ESTATE (-6)    /* call not valid in the handle's current state */
#define LBM_EIO (-7)       /* file could not be read/written, or failed its checksum */
#define LBM_ECORRUPT (-8)  /* a guard band around a device buffer was overwritten */

/* Floating-point format of the stored populations. */
#define LBM_FP64 0     /* double populations and double arithmetic */
#define LBM_FP32_DEV 1 /* float deviations f_q - t_q rho_ref, float arithmetic */

/* Viscosity modes (Sec. IV C and Eq. 10: nu = (tau_nu - 1/2) / 3). */
#define LBM_VISC_CONST 0  /* s[7], s[8] used as given */
#define LBM_VISC_STEP 1   /* nu = nu_l where rho >= rho_c, nu_v below (Sec. IV C) */
#define LBM_VISC_LINEAR 2 /* tau_nu linear in rho between rho_v and rho_l, clamped */

/* Boundaries.  x is always periodic. */
#define LBM_BC_PERIODIC 0 /* periodic in y */
#define LBM_BC_WALLS_Y 1  /* no-slip walls at y = -1/2 and y = ny - 1/2 (halfway
                             bounce-back, Sec. IV C); psi at a ghost row equals psi of the
                             adjacent fluid row */

/* Storage orientation of a batch instance (lbm_instance.layout).  The update of Eqs. 2-7
 * and 25 on a periodic lattice is symmetric under the exchange x <-> y (D2Q9 velocities,
 * force stencil weights and the moment basis map onto themselves, with j_x <-> j_y,
 * q_x <-> q_y and p_xx -> -p_xx under equal rates), so an instance may be stored and
 * swept with its axes exchanged; every host transfer of the batch converts back. */
#define LBM_LAYOUT_AUTO 0       /* transposed when that needs fewer strip rows at the
                                   batch's creation tiling (periodic instances of at least
                                   8 x 8 nodes); as given otherwise */
#define LBM_LAYOUT_ROWS 1       /* as given: rows of nx nodes */
#define LBM_LAYOUT_TRANSPOSED 2 /* axes exchanged: rows of ny nodes (periodic only) */

/* Carnahan-Starling equation of state, Eq. 30:
 *   p = rho R T (1 + x + x^2 - x^3) / (1 - x)^3 - a rho^2,  x = b rho / 4. */
typedef struct {
  double a, b, R, T;
} lbm_eos;

/* Optional settings for lbm_create.  Fill with lbm_options_default, then override. */
typedef struct {
  int precision;  /* LBM_FP32_DEV (default) or LBM_FP64 */
  int visc_mode;  /* -1 (default): LBM_VISC_STEP if nu_l > 0 and nu_v > 0, else CONST */
  int bc;         /* LBM_BC_PERIODIC (default) or LBM_BC_WALLS_Y */
  int psi_fp64;   /* FP32_DEV only: 1 evaluates psi (Eqs. 24, 30) in double precision */
  double rho_ref; /* FP32_DEV deviation reference; < 0 (default): the Maxwell vapour
                     density when T < T_c, else 0.  Ignored for LBM_FP64 (always 0). */
  double rho_c;   /* STEP switch density; <= 0 (default): 0.5218 / b (Sec. IV A) */
  double rho_l;   /* LINEAR end points; <= 0 (default): Maxwell construction (Eq. 22) */
  double rho_v;
  void* stream;   /* cudaStream_t to queue work on; NULL: a stream the handle owns */
  int device;     /* CUDA device ordinal; -1 (default): the library's current device.
                     Every call on the handle makes this device current first. */
  int tile_threads; /* threads per CTA of the step kernel; 0 (default): 128.
                       LBM_TILE_PER_INSTANCE (FP32_DEV with tile_vec 2 only): each
                       instance gets the pair-kernel width (32, 64, 96 or 128 threads)
                       that wastes least of its columns; one launch per width and kind of
                       strip per step */
  int tile_vec;     /* adjacent columns per thread: 1, or 2 (FP32 only: packed float2
                       arithmetic); available (threads, vec) pairs: FP32 (64|128|256, 1),
                       (32|64|96|128, 2); FP64 (64|128, 1).  0 (default): 2 for FP32_DEV,
                       1 for FP64.  A CTA owns threads*vec - 4 columns; with vec 2 a
                       lattice of at most 2*threads columns is swept in one full-width
                       strip per row (all threads own columns, x wraps in shared memory,
                       no ghost columns read or written). */
  int tile_rows;  /* rows per CTA sweep; 0 (default): sized to fill the GPU */
} lbm_options;

typedef struct lbm_handle lbm_handle;

/* tile_threads value: a pair-kernel width per instance (see lbm_options.tile_threads). */
#define LBM_TILE_PER_INSTANCE (-1)

/* Diagnostics of the current state (Eq. 6 fields), accumulated in double precision. */
typedef struct {
  double mass;     /* sum over nodes of rho */
  double mom_x;    /* sum over nodes of rho v_x  (rho v = sum e f + F/2, Eq. 6) */
  double mom_y;    /* sum over nodes of rho v_y */
  double max_u;    /* max over nodes of |v| (the spurious current at equilibrium) */
  double dinf;     /* max over nodes of |rho - rho at the previous diagnostics call|;
                      -1 on the first call after create/init/load */
  long long step;  /* number of steps taken since the last init */
  long long nonfinite; /* nodes whose rho or v is not finite */
} lbm_diag;

/* Fill *opt with the defaults described above.  opt must not be NULL. */
void lbm_options_default(lbm_options* opt);

/*
 * Create a lattice of nx x ny nodes (Sec. II).
 *   eos       Carnahan-Starling parameters (Eq. 30); a, b, R, T > 0.
 *   G         interaction strength of Eq. 7; must make 2 (p_EOS - rho/3) / G >= 0 over the
 *             initial densities (G = -1 in the paper, Sec. IV A).
 *   sigma     improved-forcing parameter of Eq. 25 (0 gives Eq. 9, the original scheme).
 *   s[9]      relaxation rates of Eq. 2, (s_rho, s_e, s_zeta, s_j, s_q, s_j, s_q, s_nu,
 *             s_nu), each in (0, 2).  s[1] and s[2] are the 1/tau_e and 1/tau_zeta of
 *             Eq. 25.
 *   nu_l,nu_v liquid / vapour kinematic viscosities for the STEP and LINEAR modes (> 0);
 *             they replace s[7] and s[8] there.  Pass 0, 0 for LBM_VISC_CONST.
 *   opt       NULL for defaults.
 * nx, ny >= 1 and nx*ny*9 populations must fit in device memory.  The populations start
 * at zero; call lbm_init_fields or lbm_set_populations before stepping.
 * On success *out receives the handle (free with lbm_destroy).
 */
int lbm_create(lbm_handle** out, int nx, int ny, lbm_eos eos, double G, double sigma,
               const double s[9], double nu_l, double nu_v, const lbm_options* opt);

/* Release every resource of the handle.  NULL is allowed. */
void lbm_destroy(lbm_handle* h);

/* Message of the last failure on h (NULL: of the calling thread's last failed create).
 * Never NULL; "" when there was none.  Valid until the next call on the same handle. */
const char* lbm_last_error(const lbm_handle* h);

/*
 * Set every node to the equilibrium of Eq. 3 for host fields rho, ux, uy ((ny, nx)
 * doubles; ux or uy may be NULL for zero), i.e. f_q = t_q rho [1 + 3 e.v + 9/2 (e.v)^2 -
 * 3/2 v^2].  Resets the step counter and the dinf reference.  Returns LBM_EINVAL if a
 * density is not in (0, 4/b) or gives a negative psi^2 (Eq. 24).  Synchronous.
 */
int lbm_init_fields(lbm_handle* h, const double* rho, const double* ux, const double* uy);

/* Same as lbm_init_fields from host (ny, nx) floats: half the bytes on the host link;
 * the fields are widened to double on the device before the same initialisation. */
int lbm_init_fields_f32(lbm_handle* h, const float* rho, const float* ux, const float* uy);

/* Same as lbm_init_fields with device pointers (double, (ny, nx), caller-owned). */
int lbm_init_fields_device(lbm_handle* h, const double* rho, const double* ux,
                           const double* uy);

/* Replace the state with host populations f ((9, ny, nx) doubles, pre-collision, current
 * time).  Resets the step counter.  Synchronous. */
int lbm_set_populations(lbm_handle* h, const double* f);

/* Copy the current pre-collision populations to host f ((9, ny, nx) doubles).
 * Synchronous; returns LBM_EUNSTABLE (after copying) if a step flagged a bad density. */
int lbm_get_populations(lbm_handle* h, double* f);

/*
 * Advance n >= 0 time steps (Eqs. 1-7 with the forcing of Eq. 25, Sec. II-III).  Each
 * step is one pass of the fused kernel: one launch per step, or, stepping persistently
 * (see lbm_persistent), one launch per run of up to 64 steps; runs of 64 steps are
 * replayed from a CUDA graph.
 * Asynchronous: returns once the work is queued.  Status is reported by lbm_sync and by
 * every synchronous call.
 */
int lbm_step(lbm_handle* h, int n);

/*
 * Persistent stepping (no counterpart in the paper).  With the FP32 pair kernel (tile_vec
 * 2), a run of up to 64 steps is one launch: resident CTAs take the (step, chunk row,
 * strip) work items in order from a queue, and an item waits (bounded; LBM_ETIMEOUT if it
 * runs out) only until the chunk rows whose previous step it reads, or whose previous-step
 * reads its stores would overwrite, are complete, so the CTAs of step t + 1 start while
 * step t finishes instead of the GPU draining between launches.  Results equal the
 * per-step launches bit for bit.  It is used with one kernel width (a batch's instances
 * swept in strips and those swept in full-width strips then share the launch, each work
 * item taking the sweep of its instance), at least two waves of work items per step (with
 * fewer, the first items of a step would wait on the last ones of the step before), when
 * every work item depends on at most four chunk rows (chunks of two rows or more), unless the
 * autotuner measured one launch per step faster for the tiling it chose, and unless the
 * environment sets LBM_PERSISTENT=0 when the work lists are built (creation, tiling
 * change, retirement); LBM_PERSISTENT=2 drops the two-wave condition (for tests).  With it
 * the default chunk height aims at about three waves of CTAs instead of six (taller
 * chunks, fewer halo rows: 32 rows at 4096^2).
 * lbm_persistent / lbm_batch_persistent: 1 if steps currently run that way, 0 if not,
 * LBM_EINVAL for a NULL handle.
 */
int lbm_persistent(const lbm_handle* h);

/*
 * The persistent work lists, for tests of the schedule (host code only; no device is
 * used): the step items of n_inst periodic (walls[i] == 0 or walls NULL) or walled
 * instances of nx[i] x ny[i] nodes, swept with `threads` (32, 64, 96 or 128) threads of
 * two columns and chunks of `rows` rows as one persistent work list (strips of
 * 2 threads - 4 columns, or one full-width strip per row where nx <= 2 threads, both kinds
 * in one list as in a batch's persistent launch; the library lists the strip instances
 * first, this call keeps the given order).  *n_items receives the items per
 * step; items_out (may be NULL) receives 2 n_items items, the even steps' list then the
 * odd steps', as (instance, x0, y0, y1, sweep direction), and links_out (may be NULL)
 * 2 n_items dependency links as (chunk, strips of its chunk row, four dependency chunks).
 * Returns LBM_OK, 1 if an item would depend on more than four chunks (the instances would
 * not step persistently; nothing is written), or LBM_EINVAL.
 */
int lbm_debug_persist_plan(int n_inst, const int* nx, const int* ny, const int* walls,
                           int threads, int rows, int* n_items, int* items_out,
                           int* links_out);

/* Wait for queued work, including asynchronous host transfers; LBM_EUNSTABLE if any
 * step met a non-finite or non-positive density since the last init, LBM_EINVAL if the
 * last (asynchronous) initialisation had invalid fields. */
int lbm_sync(lbm_handle* h);

/*
 * Failure-detection check (no counterpart in the paper).  Every wait of the step kernels
 * on a shared-memory copy is bounded: after a fixed number of polls the kernel gives up,
 * sets a status bit and returns, and the host reports LBM_ETIMEOUT.  This call exercises
 * that path without any device fault: a one-block kernel waits, with the same bounded-wait
 * helper, on an mbarrier that nothing arrives at, gives up after `polls` polls (1 to
 * 2^20) and sets the same status bit in the handle.  Returns LBM_ETIMEOUT; so does every
 * later lbm_sync until the state is replaced (lbm_init_fields, lbm_init_fields_device,
 * lbm_set_populations, lbm_load), after which the handle works normally.  Synchronous.
 */
int lbm_selftest_timeout(lbm_handle* h, long long polls);

/*
 * The same check for the persistent step kernel's dependency wait (see lbm_persistent):
 * one work item of the lattice is run as a two-step persistent launch whose second step
 * waits on a chunk counter that no item increments; the wait gives up after `polls`
 * rounds (1 to 2^20, each a few hundred nanoseconds), sets the timeout bit and the
 * kernel returns.  Returns LBM_ETIMEOUT, as every later lbm_sync does until the state is
 * replaced; the current state is not changed (the first step writes only the other
 * population buffer).  LBM_EINVAL unless the lattice is FP32_DEV with tile_vec 2.
 * Synchronous.
 */
int lbm_selftest_dep_timeout(lbm_handle* h, int polls);

/*
 * Discrete pressure tensor of Eq. 18 at every node of the current state (a diagnostic):
 *   P = rho c_s^2 I + (G/2) psi(x) sum_q w(|e_q|^2) psi(x + e_q) e_q e_q,
 * w = 1/3 on the axes and 1/12 on the diagonals (Eq. 7), psi of Eq. 24, rho as in
 * lbm_moments; psi beyond a wall is that of the adjacent fluid row.  With include_sigma
 * != 0 the improved forcing's extra stress is added: by Eq. 26 it is the isotropic
 * 2 G^2 sigma |grad psi|^2, evaluated with the force stencil's gradient,
 * G grad psi = -F/psi (Eq. 7), i.e. 2 sigma |F/psi|^2.  Outputs: host (ny, nx) doubles
 * pxx, pyy, pxy.  Evaluated in double precision.  Synchronous.
 */
int lbm_pressure_tensor(lbm_handle* h, double* pxx, double* pyy, double* pxy,
                        int include_sigma);

/* Density and velocity of Eq. 6 (rho v = sum e f + F/2) into host (ny, nx) doubles;
 * any pointer may be NULL.  Synchronous. */
int lbm_moments(lbm_handle* h, double* rho, double* ux, double* uy);

/* Same into host (ny, nx) floats: FP32_DEV fields as computed, FP64 fields rounded to
 * the nearest float on the device; half the bytes on the host link.  Synchronous. */
int lbm_moments_f32(lbm_handle* h, float* rho, float* ux, float* uy);

/* Same into caller-owned device arrays of (ny, nx) elements of the storage type
 * (double for LBM_FP64, float for LBM_FP32_DEV); any pointer may be NULL.  Queued on the
 * handle's stream, not synchronised. */
int lbm_moments_device(lbm_handle* h, void* rho, void* ux, void* uy);

/*
 * Asynchronous host transfers (no counterpart in the paper), for a host loop that
 * overlaps its uploads and read-backs with stepping.  The initialisation and the moments
 * pass stay in order with the steps on the handle's stream; only the host copies run on
 * two copy streams of the handle, so an upload or a read-back proceeds while earlier or
 * later steps run.  Host arrays are (ny, nx) values of the storage type (float for
 * LBM_FP32_DEV, double for LBM_FP64) and should be page-locked (cudaHostAlloc,
 * cudaHostRegister); with pageable arrays the results are the same but the copies do not
 * overlap.  Neither call waits: the caller keeps an uploaded array unchanged, and reads a
 * read-back array, only after the next lbm_sync, which waits for the copy streams too.
 *   lbm_init_fields_async: as lbm_init_fields (FP32_DEV: as lbm_init_fields_f32); ux, uy
 *     may be NULL.  The upload starts once the previous asynchronous initialisation has
 *     consumed the handle's staging buffer.  A density outside (0, 4/b), a negative psi^2
 *     or a non-finite velocity is reported as LBM_EINVAL by the next lbm_sync (or any
 *     synchronous call that reports status) unless a later initialisation replaced the
 *     state first.  The result equals lbm_init_fields(_f32) bit for bit.
 *   lbm_moments_async: as lbm_moments (FP32_DEV: as lbm_moments_f32) of the state after
 *     every step queued before the call, for the non-NULL outputs.  The next read-back,
 *     synchronous or not, waits until this one has left the handle's field buffers.
 * LBM_EINVAL for a NULL handle or rho.
 */
int lbm_init_fields_async(lbm_handle* h, const void* rho, const void* ux, const void* uy);
int lbm_moments_async(lbm_handle* h, void* rho, void* ux, void* uy);

/* Global diagnostics of the current state (see lbm_diag).  Each call also stores rho as
 * the reference of the next call's dinf.  Synchronous. */
int lbm_diagnostics(lbm_handle* h, lbm_diag* out);

/*
 * Diagnostics for callers that must not allocate device memory: a plug-in inside a host
 * application that owns the whole device-memory budget (its pool has no room, or its
 * rules forbid allocation), or a time-critical loop that cannot afford cudaMalloc and
 * cudaFree, which may synchronise the device.  The paper has no counterpart; this is the
 * lbm_diagnostics reduction with its per-CTA partial sums held in one fixed device array
 * compiled into the library (room for LBM_NOALLOC_MAX_ITEMS work items, 36 bytes each,
 * about 0.6 MB on every GPU that loads the library, kept until the process exits) instead
 * of buffers owned by the handle.
 *   out_dev  caller-owned device memory for 6 doubles per instance: mass, mom_x, mom_y,
 *            max_u, 0 (dinf is not computed: the reference density of lbm_diagnostics
 *            is neither read nor updated), count of non-finite nodes.
 * Queued on the handle's stream and not synchronised; nothing is allocated, neither on
 * the device nor on the host.  The first call on a device (and the first call after a
 * device reset, in the new context) looks up the array's device address.  All calls in
 * the process share the one array and each call overwrites it (the part it uses is
 * cleared first): calls whose work can overlap on the GPU (other streams, other handles)
 * race and must be serialised by the caller.  Returns LBM_EINVAL, with nothing queued, if the lattice needs more work items
 * than the array holds (see lbm_get_tiling; larger tiles need fewer items).
 */
#define LBM_NOALLOC_MAX_ITEMS 16384
int lbm_diagnostics_noalloc(lbm_handle* h, double* out_dev);

/* Number of steps since the last init/set/load. */
long long lbm_step_count(const lbm_handle* h);

/* psi of Eqs. 24 and 30 as the step kernel evaluates it (in the handle's precision and
 * psi mode), for n host densities; output in host doubles.  Synchronous. */
int lbm_eval_psi(lbm_handle* h, const double* rho, double* psi, size_t n);

/* Write the state (populations in storage format, parameters, step counter) to path with
 * a CRC-32; lbm_load restores it into a handle created with the same nx, ny and
 * precision (LBM_EINVAL otherwise, LBM_EIO on a short read or bad checksum). */
int lbm_save(lbm_handle* h, const char* path);
int lbm_load(lbm_handle* h, const char* path);

/* Kernel configuration in use: threads per CTA, columns per thread, rows per CTA sweep. */
int lbm_get_tiling(const lbm_handle* h, int* threads, int* vec, int* rows);
/* Change it (same meaning as the lbm_options fields; 0 picks the default). */
int lbm_set_tiling(lbm_handle* h, int threads, int vec, int rows);

/*
 * Pick the step kernel's tiling by measurement: every available (threads, vec) pair, and
 * for FP32_DEV LBM_TILE_PER_INSTANCE, with chunk heights of 1, 2, 4, 8, 12, 16, 20, 24,
 * 28, 32, 40, 48 and 64 rows is timed twice (the better time counts) over `steps` steps, rounded
 * up to even, stepped as lbm_step steps them (graph replays for each 64; CUDA events on
 * the handle's stream) on a saved copy of the state, which is restored afterwards (state and
 * step count are unchanged); a tiling that steps persistently (lbm_persistent) is timed
 * that way and again with one launch per step.  The fastest is kept, with its stepping
 * (a later lbm_set_tiling returns to the default rule).  cache_path (may be NULL) names a
 * text file of earlier choices keyed by precision, lattice sizes and GPU, one line each
 * (key, threads, vec, rows, ms per step, 1 if persistent stepping is allowed); a hit skips
 * the timing, a miss appends the new choice.  The chosen values are returned through the
 * optional out pointers (ms_per_step: the measured time of the choice, or the cached one).
 * The environment variable LBM_TILE="threads,vec,rows", when set, overrides everything.
 */
int lbm_autotune(lbm_handle* h, int steps, const char* cache_path, int* threads, int* vec,
                 int* rows, double* ms_per_step);

/* The CUDA stream the handle queues work on (a cudaStream_t). */
void* lbm_stream(const lbm_handle* h);

/*
 * Maxwell equal-area construction (Eq. 22) for the Carnahan-Starling EOS (Eq. 30):
 * coexistence densities rho_l > rho_v at temperature eos.T.  Host-only; uses the closed
 * form of int p / rho^2 d rho.  LBM_EINVAL if T is not below the critical temperature or
 * a parameter is not positive.
 */
int lbm_maxwell(lbm_eos eos, double* rho_l, double* rho_v);

/* The argument of the square root of Eq. 24 with the pressure of Eq. 30 (c = 1):
 * 2 (p_EOS(rho) - rho/3) / G, in double on the host.  psi is real where it is >= 0; the
 * kernels clamp a negative argument to zero.  LBM_EINVAL unless 0 < rho < 4/b, G != 0 and
 * the EOS parameters are positive. */
int lbm_eos_psi2(lbm_eos eos, double G, double rho, double* out);

/*
 * The coexistence densities the model selects for a flat interface: the mechanical-
 * stability condition of Eq. 21 with psi of Eq. 24 and eps = -16 G sigma (Eq. 29 with
 * alpha = 0, beta = 3), solved like lbm_maxwell (host only, no GPU).  LBM_EINVAL if T is
 * not below T_c, G >= 0, sigma < 0 or no root is bracketed.
 */
int lbm_mechanical_stability(lbm_eos eos, double G, double sigma, double* rho_l,
                             double* rho_v);

/*
 * The sigma for which Eq. 21 gives the Maxwell vapour density of eos (Eq. 22): the
 * calibration of the improved forcing against thermodynamics (Sec. IV A-B): a scan of
 * sigma = 0.01, 0.02, .. 0.5 for the first sign change between two values at which Eq. 21
 * has a solution, then bisection.  Host only.  LBM_EINVAL if there is none (Eq. 21 has
 * no positive-pressure solution for small sigma at low reduced temperatures).
 */
int lbm_sigma_consistent(lbm_eos eos, double G, double* sigma);

/* ---------------------------------------------------------------------------------- */
/* Batches: many independent lattices (uneven sizes, own EOS and rates) advanced by one
 * kernel launch per step. */

typedef struct lbm_batch lbm_batch;

/* One instance of a batch; the fields mean what the lbm_create arguments mean. */
typedef struct {
  int nx, ny;
  lbm_eos eos;
  double G, sigma;
  double s[9];
  double nu_l, nu_v;
  int visc_mode;   /* LBM_VISC_* (no automatic choice here) */
  int bc;          /* LBM_BC_* */
  double rho_c;    /* <= 0: 0.5218 / b */
  double rho_l;    /* <= 0: Maxwell */
  double rho_v;
  double rho_ref;  /* < 0: Maxwell vapour density (FP32_DEV only) */
  int layout;      /* LBM_LAYOUT_* (0, the zero-initialised value, is AUTO).  A transposed
                      instance is stepped as the ny x nx lattice with the axes exchanged;
                      lbm_batch_init_fields*, lbm_batch_moments*,
                      lbm_batch_get_populations and lbm_batch_diagnostics take and return
                      its fields, populations and momentum in the given (nx, ny)
                      orientation, so the layout is visible only through
                      lbm_batch_instance_transposed and the rounding of the results (a
                      transposed instance equals, bit for bit, the ny x nx lattice started
                      from the transposed fields).  TRANSPOSED with LBM_BC_WALLS_Y is
                      LBM_EINVAL. */
} lbm_instance;

/* Create a batch of n >= 1 instances in one precision; stream may be NULL; device,
 * tile_threads, tile_vec and tile_rows as in lbm_options (-1, 0, 0, 0 = defaults).  The
 * orientation of each LBM_LAYOUT_AUTO instance is fixed here, from the strip rows of its
 * two orientations at this tiling (a strip row of w computed columns costing w + 57
 * column-equivalents; the pair-kernel width rule under LBM_TILE_PER_INSTANCE), and kept
 * through later tiling changes. */
int lbm_batch_create(lbm_batch** out, int n, const lbm_instance* inst, int precision,
                     void* stream, int device, int tile_threads, int tile_vec,
                     int tile_rows);
void lbm_batch_destroy(lbm_batch* b);
const char* lbm_batch_last_error(const lbm_batch* b);

/* Equilibrium initialisation of instance i from host fields, as lbm_init_fields. */
int lbm_batch_init_fields(lbm_batch* b, int i, const double* rho, const double* ux,
                          const double* uy);
/* Advance every active instance n steps (one launch per step, kernel width and kind of
 * strip, or one per run of up to 64 steps stepping persistently; CUDA-graph replay; see
 * lbm_batch_launches_per_step and lbm_batch_persistent). */
int lbm_batch_step(lbm_batch* b, int n);
/* Float host variant of lbm_batch_init_fields, as lbm_init_fields_f32. */
int lbm_batch_init_fields_f32(lbm_batch* b, int i, const float* rho, const float* ux,
                              const float* uy);
/* Host moments of instance i, as lbm_moments (lbm_batch_moments_f32: as lbm_moments_f32). */
int lbm_batch_moments(lbm_batch* b, int i, double* rho, double* ux, double* uy);
int lbm_batch_moments_f32(lbm_batch* b, int i, float* rho, float* ux, float* uy);
/* Host populations of instance i, as lbm_get_populations. */
int lbm_batch_get_populations(lbm_batch* b, int i, double* f);
/* Per-instance diagnostics (out has n entries), as lbm_diagnostics. */
int lbm_batch_diagnostics(lbm_batch* b, lbm_diag* out);

/*
 * Step until every instance is converged: an instance converges at the first check
 * where max |rho - rho 'check_every' steps earlier| < tol, after which it stops being
 * stepped (its state is frozen).  An instance whose state turns non-finite or
 * non-positive is retired at the next check the same way (it does not converge; its
 * diagnostics keep reporting the non-finite nodes).  Checks run every check_every steps;
 * at most max_steps steps are taken.  steps_out (n entries, may be NULL) receives each
 * instance's step count at convergence, or -1 if it did not converge.  Returns the number
 * of instances still being stepped (neither converged nor retired; >= 0) or a negative
 * error.
 */
int lbm_batch_run_to_equilibrium(lbm_batch* b, double tol, int check_every,
                                 long long max_steps, long long* steps_out);

/* Number of instances still being stepped. */
int lbm_batch_active(const lbm_batch* b);
/* 1 if instance i is stored transposed (lbm_instance.layout), 0 if as given, LBM_EINVAL
 * for a bad handle or index. */
int lbm_batch_instance_transposed(const lbm_batch* b, int i);
/* 1 if instance i is still being stepped, 0 if it is frozen (converged or retired),
 * LBM_EINVAL for a bad handle or index. */
int lbm_batch_instance_active(const lbm_batch* b, int i);

/*
 * Retirement of instances that are no longer to be stepped (a batch-runtime service; the
 * paper has none).  lbm_batch_retire freezes instance i as convergence does: its state
 * stays as it is, later steps and graph replays skip it, and lbm_batch_init_fields (or
 * its float form) makes it active again.  lbm_batch_retire_nonfinite runs the
 * diagnostics pass (as lbm_batch_diagnostics: synchronous, and it sets the reference of
 * the next dinf) and retires every active instance that has a non-finite
 * or non-positive density, so that the rest of the batch is stepped (and timed) without
 * it; retired (n entries, may be NULL) receives 1 for each instance it retired, 0
 * otherwise.  Returns the number retired (>= 0) or a negative error.
 */
int lbm_batch_retire(lbm_batch* b, int i);
int lbm_batch_retire_nonfinite(lbm_batch* b, int* retired);

/* lbm_autotune for a batch (all active instances are stepped together). */
int lbm_batch_autotune(lbm_batch* b, int steps, const char* cache_path, int* threads,
                       int* vec, int* rows, double* ms_per_step);
/* Tiling in use by a batch (threads is LBM_TILE_PER_INSTANCE for per-instance widths). */
int lbm_batch_get_tiling(const lbm_batch* b, int* threads, int* vec, int* rows);
/* Step-kernel launches of lbm_batch_step per step (0 when nothing is active): one per
 * launch group, that is per kernel width in use (several only with LBM_TILE_PER_INSTANCE)
 * and kind of strip (full-width strips for instances of at most 2 * threads columns,
 * strips for wider ones; pair kernel only); 1 when the batch steps persistently
 * (lbm_batch_persistent), every group then sharing one launch per run of up to 64 steps. */
int lbm_batch_launches_per_step(const lbm_batch* b);
/* Persistent stepping of a batch (see lbm_persistent). */
int lbm_batch_persistent(const lbm_batch* b);

/*
 * Integrity checks and fault injection (for tests of the library and of its callers).
 *
 * The population slabs, the moment fields, the previous-density array and the host
 * staging buffer of a handle are allocated with 4096-byte guard bands of a fixed byte
 * pattern on each side.  lbm_check_guards (lbm_batch_check_guards) synchronises the
 * handle's stream and reads them back: LBM_OK while every guard byte is intact,
 * LBM_ECORRUPT (the message names the buffer and the offset) if any kernel or copy wrote
 * outside its buffer.
 */
int lbm_check_guards(lbm_handle* h);
int lbm_batch_check_guards(lbm_batch* b);

/*
 * lbm_debug_fail_alloc(n), n >= 0: the next n device allocations made by lattice and
 * batch handles (process-wide) succeed and the one after fails, as an out-of-memory
 * would (the call that made it returns LBM_ENOMEM and releases what it had allocated);
 * the hook then disarms itself.  n < 0 disarms it.  Returns the previous setting.
 */
int lbm_debug_fail_alloc(int n);

/* 1 in the bounds-check build of the library (kernels compiled with LBM_BOUNDS_CHECK:
 * every global and shared-memory access of the step kernels is index-checked; an access
 * that fails its check is skipped and the next status check returns LBM_ECORRUPT), 0 in
 * the normal build. */
int lbm_bounds_checked(void);

/* Device allocations made by lattice and batch handles and not yet released
 * (process-wide): returns to its earlier value once every handle created since is
 * destroyed, whether or not its calls failed. */
long long lbm_debug_live_allocs(void);

/*
 * Overwrite one byte of the guard band just after guarded buffer `which` of the handle
 * (0 and 1: the population slabs, 2: the previous density), so that lbm_check_guards
 * must report it.  A host-side copy into memory the handle owns: no kernel runs and
 * nothing outside the allocation is touched.  LBM_EINVAL for an unknown buffer.
 */
int lbm_debug_corrupt_guard(lbm_handle* h, int which);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
