/*
 * mptrac.h -- C ABI of the GB300 Lagrangian transport hot path.
 *
 * The calls follow the structure of the MPTRAC time loop described in
 * arxiv 2211.12616:
 *   mptrac_load_met   ~ read_met + "update device" of a met snapshot (Sections 3.1, 4.1)
 *   mptrac_set_releases / release masking ~ module_timesteps       (Section 4.3)
 *   mptrac_advect     ~ module_advection + module_position          (Section 3.2)
 *   mptrac_diffuse    ~ module_diffusion_turb + module_diffusion_meso with
 *                       per-device counter-based random numbers     (Sections 3.2, 4.3)
 *   mptrac_step       ~ the fused chain advection -> turbulent -> mesoscale
 *                       diffusion -> position, as called in the time loop
 *   mptrac_sort       ~ the particle sorting modules                (Section 6)
 *   mptrac_step_sort  ~ mptrac_step then mptrac_sort, fused through the sort workspace
 * The paper prints no formulas for any of these; the numerics implemented are:
 *   - 4D linear interpolation (lon periodic, lat clamped, linear in p between
 *     levels, linear in time between two snapshots);
 *   - explicit midpoint step on the sphere, R = 6371 km, angles in degrees,
 *     second stage with cos(lat) of the midpoint;
 *   - turbulent diffusion sqrt(2 D dt) xi (horizontal metres; vertical metres
 *     converted as dp = -p dz / H);
 *   - mesoscale AR(1) wind perturbation scaled by the subgrid standard
 *     deviation: on each snapshot the spread of the 8 cell-corner winds about
 *     the interpolated wind, weighted by the interpolation weights, then
 *     linear in time;
 *   - Philox4x32-10 (Salmon et al., SC'11) with counter
 *     (particle id, step, stream, release), key = seed, Box-Muller normals;
 *     the normals of stream 0 then stream 1 are used in order (turbulence
 *     z0..z2 of stream 0, mesoscale z3 of stream 0 and z0, z1 of stream 1);
 *   - lat reflected over the poles (lon + 180), lon wrapped into
 *     [lon0, lon0 + 360), p clamped to the level range.
 *
 * Conventions
 *   - Every function returns an int status (MPTRAC_OK = 0, negative = error);
 *     mptrac_last_error() gives a message for the calling thread's last error.
 *     No C++ exception crosses this boundary.  Arguments are validated on the
 *     host before anything is launched; an invalid call launches nothing.
 *   - "device" pointers are CUDA device (or managed) memory owned by the caller;
 *     the library never frees them.  "host" pointers are read before the call
 *     returns unless stated otherwise.
 *   - Work is enqueued asynchronously on `stream` (a cudaStream_t passed as an
 *     integer; 0 = legacy default stream).  Results are ready once the stream
 *     has been synchronised.  There is no CPU fallback: without a usable CUDA
 *     device every call that launches work returns MPTRAC_E_CUDA.
 *   - A context is not thread-safe; calls on one context must be serialised
 *     by the caller (they may use different streams).
 *   - A context (and a surrogate) lives on the device that was current when it
 *     was created; every call on it makes that device current for its duration
 *     and restores the caller's.  `stream` must belong to that device.
 */
#ifndef MPTRAC_H
#define MPTRAC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define MPTRAC_OK              0
#define MPTRAC_E_INVALID_ARG  -1   /* a pointer, size or parameter is invalid */
#define MPTRAC_E_OOM          -2   /* device allocation failed */
#define MPTRAC_E_CUDA         -3   /* a CUDA runtime call or launch failed */
#define MPTRAC_E_TIME_RANGE   -4   /* [t, t + nsteps*dt] lies in no interval of the loaded snapshots */
#define MPTRAC_E_WORKSPACE    -5   /* workspace pointer NULL, misaligned or too small */
#define MPTRAC_E_TIMEOUT      -6   /* a bounded device-side wait gave up (reported by mptrac_surr_status) */
#define MPTRAC_E_NOT_INIT     -7   /* context NULL, or met snapshots not loaded */

/* ---- met storage precision -------------------------------------------- */
#define MPTRAC_FP32 0   /* 4 x float32 per grid point */
#define MPTRAC_BF16 1   /* 4 x bfloat16 codes + per-(level,variable) power-of-two scale */
#define MPTRAC_FP16 2   /* 4 x float16 codes + per-(level,variable) power-of-two scale */

#define MPTRAC_MAX_NZ        256   /* largest supported number of pressure levels */
#define MPTRAC_NUM_SLOTS       3   /* met slots of a context */
#define MPTRAC_MAX_RELEASES  65536 /* largest release table */

typedef struct mptrac_ctx mptrac_ctx;   /* opaque: met slots, level tables, release table */

/* Grid of the met snapshots (the paper's met_t, Section 3.1).
 *   nx, ny, nz      number of longitudes, latitudes and pressure levels
 *                   (nx >= 2, ny >= 2, 2 <= nz <= MPTRAC_MAX_NZ)
 *   lon0, dlon      first longitude and spacing [deg]; the grid is periodic:
 *                   nx * dlon must equal 360 (within 1e-9)
 *   lat0, dlat      first latitude and spacing [deg], dlat > 0
 *   plev            HOST array of nz levels [Pa], strictly decreasing
 *                   (level 0 is the lowest); copied during the call
 *   storage         MPTRAC_FP32 / MPTRAC_BF16 / MPTRAC_FP16
 *   nvars           3 (u, v, omega) or 4 (u, v, omega, T)                  */
typedef struct {
    int nx, ny, nz;
    double lon0, dlon, lat0, dlat;
    const double* plev;
    int storage;
    int nvars;
} mptrac_grid_desc;

/* Particle state (the paper's atm_t, Section 4.4), structure of arrays of
 * length n (0 <= n <= 2^31 - 1; every call rejects other counts with
 * E_INVALID_ARG), all DEVICE pointers owned by the caller.
 *   lon, lat, p     float64 positions [deg, deg, Pa]; lon in [lon0, lon0+360)
 *   id              uint32 particle identity (the random-number counter uses
 *                   it, so results do not depend on the array order)
 *   release         uint32 release index into the table set by
 *                   mptrac_set_releases, or NULL (all particles always active)
 *   up, vp, wp      float32 mesoscale wind perturbations [m/s, m/s, Pa/s];
 *                   may be NULL when mesoscale diffusion is off and the arrays
 *                   are not to be sorted.                                    */
typedef struct {
    int64_t n;
    double* lon;
    double* lat;
    double* p;
    uint32_t* id;
    uint32_t* release;
    float* up;
    float* vp;
    float* wp;
} mptrac_particles;

/* Diffusion parameters (module_diffusion_turb / module_diffusion_meso).
 *   dx, dz          horizontal and vertical turbulent diffusivity [m^2/s], >= 0
 *   meso_f          mesoscale scaling factor f, >= 0
 *   scale_height    H [m] converting vertical metres to pressure, > 0
 *   turb, meso      non-zero to enable each term                          */
typedef struct {
    double dx, dz;
    double meso_f;
    double scale_height;
    int turb, meso;
} mptrac_diff_params;

/* Creates a context for grid `g`: allocates MPTRAC_NUM_SLOTS (3) device met
 * slots, their interleaved copies (for every pair of slots, both slots' values
 * of a grid point in one record, the layout the particle kernels gather from;
 * each as large as two slots) and the level tables on the current CUDA device.
 * Two slots hold a met interval; the third lets the next snapshot be loaded
 * while the current interval is being used.  On success *out owns them until
 * mptrac_destroy.  Errors: E_INVALID_ARG (bad grid), E_OOM, E_CUDA. */
int mptrac_init_grid(mptrac_ctx** out, const mptrac_grid_desc* g);

/* Frees everything the context owns (after synchronising the device). NULL is a no-op. */
int mptrac_destroy(mptrac_ctx* ctx);

/* Message of the calling thread's most recent error ("" if none). `ctx` may be NULL. */
const char* mptrac_last_error(const mptrac_ctx* ctx);

/* Loads snapshot time `t` [s] into met slot `slot` (0, 1 or 2)  -- read_met +
 * update device (Sections 3.1, 4.1).  u, v, omega (and T when nvars == 4,
 * otherwise ignored) are float32 arrays of nz*ny*nx values in layout
 * [level][lat][lon], on the DEVICE if src_is_device != 0, else on the HOST (copied
 * on `stream` through a context-owned staging buffer; the host arrays must
 * stay valid until the stream has passed this call).  The slot is rewritten
 * as records [lat][lon][level] x (u, v, omega, T) in the grid's storage
 * precision; reduced precision uses per-(level, variable) power-of-two scales
 * 2^(E-15), maxabs = m 2^E, m in [0.5, 1).  The same values are written to
 * this slot's lane of the interleaved copies it belongs to (never the copy of
 * the other two slots, so a load does not disturb work in flight on them).
 * Every call that interpolates in time uses the two loaded slots that are
 * consecutive in time and whose interval contains its time range (the earlier
 * one is the interval start): E_NOT_INIT if fewer than two slots with
 * different times are loaded, E_TIME_RANGE if no such interval contains it.
 * Errors: E_INVALID_ARG, E_NOT_INIT, E_CUDA. */
int mptrac_load_met(mptrac_ctx* ctx, int slot, double t,
                    const float* u, const float* v, const float* omega, const float* T,
                    int src_is_device, uintptr_t stream);

/* Release table for time-step masking (module_timesteps, Section 4.3):
 * a particle of release r moves at step time t_n only if
 * t_start[r] <= t_n < t_end[r].  HOST arrays of n entries (0 < n <=
 * MPTRAC_MAX_RELEASES), copied synchronously.  n == 0 clears the table (then
 * every particle is active whatever its release index).
 * Particles whose release index is >= n are never active. */
int mptrac_set_releases(mptrac_ctx* ctx, int n, const double* t_start, const double* t_end);

/* nsteps explicit midpoint advection steps from time t with step dt > 0
 * (module_advection, each step followed by module_position).  Requires
 * t0 <= t and t + nsteps*dt <= t1 for the loaded snapshot times, else
 * E_TIME_RANGE.  nsteps >= 0.  Particle positions are updated in place. */
int mptrac_advect(mptrac_ctx* ctx, const mptrac_particles* parts, double t, double dt,
                  int nsteps, uintptr_t stream);

/* nsteps diffusion-only steps (module_diffusion_turb + module_diffusion_meso +
 * module_position): subgrid variance and displacement at the current position.
 * Random numbers: Philox4x32-10, counter (id, step0 + n, stream 0|1, release)
 * with the low 32 bits of step0 + n (the draws repeat after 2^32 steps),
 * key (seed low, seed high words).  up/vp/wp must be non-NULL when
 * prm->meso != 0.  Same time-range rule as mptrac_advect. */
int mptrac_diffuse(mptrac_ctx* ctx, const mptrac_particles* parts, double t, double dt,
                   const mptrac_diff_params* prm, uint64_t seed, uint64_t step0,
                   int nsteps, uintptr_t stream);

/* Fused production step: per step, midpoint advection (its first wind
 * evaluation also yields the corner variances), turbulent + mesoscale
 * displacement converted at the post-advection position, then the position
 * rules.  With prm->turb == prm->meso == 0 it equals mptrac_advect; with a
 * zero wind it equals mptrac_diffuse.  The particle state stays in registers
 * for all nsteps steps of the call (temporal blocking). */
int mptrac_step(mptrac_ctx* ctx, const mptrac_particles* parts, double t, double dt,
                const mptrac_diff_params* prm, uint64_t seed, uint64_t step0,
                int nsteps, uintptr_t stream);

/* Bytes of device workspace mptrac_sort needs for n particles. */
size_t mptrac_sort_workspace_bytes(const mptrac_ctx* ctx, int64_t n);

/* Sorts the particles by met cell (Section 6, the sorting modules): key =
 * (j*nx + i)*nz + k of the cell containing each particle (same cell rule as
 * the interpolation), stable LSD radix sort, then every non-NULL array of
 * `parts` is permuted the same way.  `workspace` is caller-owned DEVICE memory,
 * 256-byte aligned, of at least mptrac_sort_workspace_bytes(ctx, n) bytes,
 * else E_WORKSPACE.  It must not be in use by another call in flight. */
int mptrac_sort(mptrac_ctx* ctx, const mptrac_particles* parts, void* workspace,
                size_t ws_bytes, uintptr_t stream);

/* mptrac_step followed by mptrac_sort, with the same result, fused: the step's
 * last launch writes each particle's final state to the sort workspace
 * together with its cell key and the first radix digit's histogram, so the
 * sort reads no particle array again (the time loop of Sections 3-4 with the
 * sorting modules of Section 6).  The paper has no such call; it saves a pass
 * over the particles per sort.  Arguments and errors as mptrac_step and
 * mptrac_sort (workspace rules included); with nsteps == 0 it is mptrac_sort.
 * It is mptrac_step_handoff followed by mptrac_sort_handoff. */
int mptrac_step_sort(mptrac_ctx* ctx, const mptrac_particles* parts, double t, double dt,
                     const mptrac_diff_params* prm, uint64_t seed, uint64_t step0, int nsteps,
                     void* workspace, size_t ws_bytes, uintptr_t stream);

/* First half of mptrac_step_sort: the steps, with the final state left in
 * `workspace` (with the cell keys) and the arrays of `parts` NOT updated.
 * Until mptrac_sort_handoff has run on the same workspace and particles, the
 * particle arrays hold the state before the call.  nsteps >= 1, else
 * E_INVALID_ARG; otherwise arguments and errors as mptrac_step_sort. */
int mptrac_step_handoff(mptrac_ctx* ctx, const mptrac_particles* parts, double t, double dt,
                        const mptrac_diff_params* prm, uint64_t seed, uint64_t step0, int nsteps,
                        void* workspace, size_t ws_bytes, uintptr_t stream);

/* Second half of mptrac_step_sort: radix sort of the keys a preceding
 * mptrac_step_handoff left in `workspace`, gathering the final state into the
 * arrays of `parts` in sorted order.  Calling it without that hand-off leaves
 * garbage in `parts`. */
int mptrac_sort_handoff(mptrac_ctx* ctx, const mptrac_particles* parts, void* workspace,
                        size_t ws_bytes, uintptr_t stream);

/* module_meteo (Section 3.2): u, v, omega and T (0 when nvars == 3) at every
 * particle position at time t, by the 4D linear interpolation of the
 * advection (float32 arithmetic), into DEVICE out[4][n] (variable-major).
 * t must lie within the loaded snapshots (E_TIME_RANGE). */
int mptrac_sample_met(mptrac_ctx* ctx, const mptrac_particles* parts, double t, float* out,
                      uintptr_t stream);

/* module_sedi (Section 3.2): nsteps sedimentation steps from time t.  Spherical
 * particles of radius[i] [m] and density[i] [kg/m^3] (DEVICE float32 arrays of
 * n) settle at the Stokes velocity with the Cunningham slip correction,
 * v_s = 2 r^2 (rho_p - rho_air) g C / (9 eta), C = 1 + Kn (1.257 + 0.4 e^(-1.1/Kn)),
 * Kn = 2 eta / (rho_air vbar r), vbar = sqrt(8 R_d T / pi), eta by Sutherland's
 * formula, rho_air = p / (R_d T), with T interpolated at the particle; the
 * fall is dp = rho_air g v_s dt (p clamped).  Needs nvars == 4. */
int mptrac_sediment(mptrac_ctx* ctx, const mptrac_particles* parts, const float* radius,
                    const float* density, double t, double dt, int nsteps, uintptr_t stream);

/* write_grid (Section 3.3) for particle counts: the number of particles in every
 * met cell, indexed by the cell key of mptrac_sort ((j*nx + i)*nz + k), into
 * DEVICE counts[nx*ny*nz] (overwritten; cells of the last latitude row or the
 * top level are never used by the cell rule and stay zero). */
int mptrac_grid_counts(mptrac_ctx* ctx, const mptrac_particles* parts, uint32_t* counts,
                       uintptr_t stream);

/* Sort for runs with a release table: as mptrac_sort, except that particles
 * whose release is not active at time t (t outside [t_start, t_end) of its
 * release, or a release index outside the table) are keyed after every cell,
 * so active particles fill the front of the arrays and whole warps of the
 * step kernel work on active particles.  Equal keys keep their order.  Without
 * a release table, or with parts->release == NULL, this is mptrac_sort. */
int mptrac_sort_at(mptrac_ctx* ctx, const mptrac_particles* parts, double t, void* workspace,
                   size_t ws_bytes, uintptr_t stream);

/* Launch configuration of the fused step kernel (a project tuning knob; the
 * paper has none).  Results do not depend on it.
 *   variant     0: 256 threads per block, >= 2 resident blocks per SM (128 registers)
 *               1: 128 threads per block, >= 4 resident blocks per SM (128 registers)
 *               2: 128 threads per block, >= 5 resident blocks per SM (96 registers)
 *               3: 128 threads per block, >= 6 resident blocks per SM (80 registers),
 *                  the per-particle corner cache in shared memory (24.6 KB per block)
 *               4: as 3 with >= 7 resident blocks per SM (72 registers)
 *               5: 64 threads per block, >= 10 resident blocks per SM (96 registers)
 *               6: 512 threads per block, >= 1 resident block per SM (128 registers)
 *   schedule    0: one thread per particle (the default);
 *               1: one wave of blocks (SMs x resident blocks per SM) strides over
 *                  the particles;
 *               k in 2..64: k particles per thread (ceil(n / (threads per block x k))
 *                  blocks stride over the particles).
 * Both apply to the fused step with diffusion (mptrac_step and the forms that end in
 * a sort hand-off); the other transport calls (advection only, diffusion only,
 * masked advection) keep one fixed launch shape.
 * Errors: E_INVALID_ARG for an unknown variant or a schedule outside 0..64. */
int mptrac_set_launch(mptrac_ctx* ctx, int variant, int schedule);

/* Sort without any device allocation.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory (a host
 * that must not bypass another framework's pool allocator, a pipeline in which
 * cudaMalloc's implicit device synchronisation is not allowed, or a process
 * with a device memory budget fixed at start-up).  It does what mptrac_sort
 * does, with the same result, but its scratch memory is a 16 MiB array that is
 * part of the library image (held by every GPU that loads the library until
 * exit) instead of a caller workspace; it calls no allocating routine.
 *   - At most MPTRAC_SORT_NOALLOC_MAX_N particles, else E_INVALID_ARG
 *     (nothing is launched).
 *   - The first call on a device looks up the array's device address on that
 *     (current) device; make that first call before any stream capture.
 *   - All calls on one device share the array: calls that overlap on the GPU
 *     race and must be serialised by the caller.
 * Errors: as mptrac_sort (without E_WORKSPACE for a missing workspace). */
#define MPTRAC_SORT_NOALLOC_MAX_N 262144
int mptrac_sort_noalloc(mptrac_ctx* ctx, const mptrac_particles* parts, uintptr_t stream);

/* ---- learned displacement surrogate (the project's addition; the paper has
 * no learned component) -----------------------------------------------------
 * A small MLP maps a particle's local wind stencil to its displacement over
 * one 30-minute segment (10 plain midpoint substeps of 180 s):
 *   features (MPTRAC_SURR_NFEAT = 168, zero-padded to MPTRAC_SURR_KPAD = 176):
 *     u, v, omega at the 3x3x3 grid nodes around the nearest node on both
 *     snapshots, ordered [snapshot][variable][dk][dj][di]; the offsets of the
 *     position from that node in grid units (lon, lat, fractional level); the
 *     time weight; sin(lat), cos(lat);
 *   x_hat = (x - mu_x)/sd_x, z1 = x_hat W1 + b1, h1 = gelu(z1), z2 = h1 W2 + b2,
 *   h2 = gelu(z2), y_hat = h2 W3 + b3, y = y_hat sd_y + mu_y, with
 *   gelu(x) = x/2 (1 + erf(x/sqrt 2));
 *   outputs: east and north displacement [m] at the start latitude, ln(p1/p0).
 * Parameters: one float32 vector of MPTRAC_SURR_NPARAM values laid out as
 * W1 [176][128] (row-major, rows 168..175 unused), b1 [128], W2 [128][128],
 * b2 [128], W3 [128][3], b3 [3].  GEMMs run on tensor cores in bfloat16 with
 * float32 accumulation; loss, biases and Adam in float32. */
#define MPTRAC_SURR_NFEAT   168
#define MPTRAC_SURR_KPAD    176
#define MPTRAC_SURR_HIDDEN  128
#define MPTRAC_SURR_NOUT    3
#define MPTRAC_SURR_NPARAM  39555

typedef struct mptrac_surr mptrac_surr;   /* opaque: parameters, Adam state, activations */

/* Creates a surrogate able to process up to max_batch samples per call (device
 * buffers sized for it); parameters, Adam moments and the normalisation start
 * at zero / identity. */
int mptrac_surr_create(mptrac_surr** out, int64_t max_batch);
int mptrac_surr_destroy(mptrac_surr* s);
/* HOST arrays of MPTRAC_SURR_NPARAM floats (copied synchronously). */
int mptrac_surr_set_params(mptrac_surr* s, const float* params);
int mptrac_surr_get_params(const mptrac_surr* s, float* params);
/* Gradients of the last mptrac_surr_grads / mptrac_surr_train_step (HOST out). */
int mptrac_surr_get_grads(const mptrac_surr* s, float* grads);
/* Feature and target normalisation, HOST arrays: mu_x, sd_x of KPAD entries
 * (entries >= NFEAT ignored), mu_y, sd_y of NOUT entries; sd > 0. */
int mptrac_surr_set_norm(mptrac_surr* s, const float* mu_x, const float* sd_x, const float* mu_y,
                         const float* sd_y);
/* Raw features of every particle at time t (t within the loaded snapshots)
 * into DEVICE feat [n][KPAD].  Grid needs nx, ny, nz >= 3. */
int mptrac_surr_features(mptrac_ctx* ctx, const mptrac_particles* parts, double t, float* feat,
                         uintptr_t stream);
/* Targets from start and end positions (DEVICE float64 arrays of n) into
 * DEVICE y [n][NOUT]: dx = R cos(lat0) dlon, dy = R dlat (radians, dlon folded
 * into [-180, 180) degrees), dz = ln(p1/p0). */
int mptrac_surr_targets(int64_t n, const double* lon0, const double* lat0, const double* p0,
                        const double* lon1, const double* lat1, const double* p1, float* y,
                        uintptr_t stream);
/* Column means and standard deviations of DEVICE data [n][ncol] (float32,
 * n >= 1, ncol <= 4096) into DEVICE mean[ncol], sd[ncol] (float64): sums in
 * float32 per block of rows (compensated) and in float64 across blocks, then
 * sd = sqrt(max(sum of squares / n - mean^2, 0)).  An sd not above sd_min is
 * written as 1, so that a constant column (a padding feature) standardises to
 * zero.  The statistics the surrogate's standardisation takes (training). */
int mptrac_surr_colstats(const float* data, int64_t n, int ncol, double* mean, double* sd,
                         double sd_min, uintptr_t stream);
/* Normalised outputs y_hat of n <= max_batch DEVICE raw feature rows into
 * DEVICE y_hat [n][8] (columns 3..7 are zero padding). */
int mptrac_surr_forward(mptrac_surr* s, const float* x, int64_t n, float* y_hat, uintptr_t stream);
/* Loss (mean squared error in normalised units, ADDED to DEVICE *loss) and
 * gradients for n <= max_batch samples (DEVICE x [n][KPAD], y [n][NOUT] raw). */
int mptrac_surr_grads(mptrac_surr* s, const float* x, const float* y, int64_t n, float* loss,
                      uintptr_t stream);
/* mptrac_surr_grads followed by one Adam step (beta1 0.9, beta2 0.999,
 * eps 1e-8, bias correction with step >= 1) at learning rate lr. */
int mptrac_surr_train_step(mptrac_surr* s, const float* x, const float* y, int64_t n, float lr,
                           int step, float* loss, uintptr_t stream);
/* One epoch of training in a single call: floor(n / batch) Adam steps, as
 * mptrac_surr_train_step, on the consecutive mini-batches x[b batch ...],
 * y[b batch ...] (DEVICE, as for mptrac_surr_grads; the caller shuffles), with
 * step numbers step0 + 1, step0 + 2, ... and the cosine learning-rate decay
 *     lr(step) = lr_min + (lr_max - lr_min) (1 + cos(pi step / total_steps)) / 2
 * evaluated in float64 (in this order, without fused multiply-adds) and
 * rounded to float32 (lr_max at step 0, lr_min at step total_steps).  Each
 * batch's loss is ADDED to DEVICE *loss.  The result equals the same steps
 * made one call at a time.  Rows past the last whole batch are not used.  Errors: E_INVALID_ARG for batch outside [1, max_batch],
 * n < batch, lr_min <= 0 or lr_max < lr_min, steps outside [1, total_steps], or
 * host pointers; nothing is launched then. */
int mptrac_surr_train_epoch(mptrac_surr* s, const float* x, const float* y, int64_t n, int64_t batch,
                            double lr_max, double lr_min, int step0, int total_steps, float* loss,
                            uintptr_t stream);
/* One 30-minute surrogate segment from time t (segment length dt_seg [s]):
 * particles inside the training envelope (|lat| <= 80 deg, every standardised
 * feature within +-4, [t, t + dt_seg] inside the loaded snapshots) move by
 * the predicted displacement followed by the position rules; the others are
 * left in place with fallback[i] = 1 (DEVICE uint8 [n]) for the plain
 * integrator (mptrac_advect_masked).  If fallback_count (DEVICE uint64) is not
 * NULL, the number of particles flagged is ADDED to it.  Any n. */
int mptrac_surr_advance(mptrac_ctx* ctx, mptrac_surr* s, const mptrac_particles* parts, double t,
                        double dt_seg, uint8_t* fallback, uint64_t* fallback_count, uintptr_t stream);
/* Tensor-core kernels of the surrogate (training GEMMs and the fused
 * inference in mptrac_surr_advance):
 *   MPTRAC_SURR_KERNEL_TCGEN05 (default): tcgen05.mma chains issued by one
 *     thread per CTA (M = 128, K in steps of 16), operands in shared memory,
 *     accumulators in tensor memory;
 *   MPTRAC_SURR_KERNEL_MMA_SYNC: warp-level mma.sync m16n8k16, kept for
 *     comparison.
 *   MPTRAC_SURR_KERNEL_WAIT_TEST: the tcgen05 kernel with its MMAs withheld
 *     and a wait limit of about 10 ms, for tests of the bounded wait: nothing
 *     moves and mptrac_surr_status reports E_TIMEOUT.
 * Both compute the same network in bf16 with float32 accumulation and add
 * the K = 16 products in the same order: the inference results have been
 * identical, the gradients differ by the grouping of their split-K atomic
 * sums.  E_INVALID_ARG for another value. */
#define MPTRAC_SURR_KERNEL_TCGEN05   0
#define MPTRAC_SURR_KERNEL_MMA_SYNC  1
#define MPTRAC_SURR_KERNEL_WAIT_TEST 2
int mptrac_surr_set_kernel(mptrac_surr* s, int kernel);
/* Synchronises `stream` and reports whether a tcgen05 kernel of this surrogate
 * launched before gave up a bounded wait for its tensor-core work (about one
 * second):
 * E_TIMEOUT (the flag is then cleared; after an inference the particles of
 * the tiles not reached are left unmoved and their fallback entries are not
 * written, after a training call the gradients are incomplete), else OK. */
int mptrac_surr_status(mptrac_surr* s, uintptr_t stream);
/* mptrac_advect restricted to particles with mask[i] != 0 (DEVICE uint8 [n]). */
int mptrac_advect_masked(mptrac_ctx* ctx, const mptrac_particles* parts, const uint8_t* mask,
                         double t, double dt, int nsteps, uintptr_t stream);

/* ---- inspection entry points (used by the parity tests) ---------------- */

/* Cell keys of the sort, written to DEVICE array keys[n]. */
int mptrac_cell_keys(mptrac_ctx* ctx, const mptrac_particles* parts, uint32_t* keys,
                     uintptr_t stream);

/* Wind (u, v, omega) interpolated at n DEVICE positions lon/lat/p (float64)
 * and time t (4D linear, float32 arithmetic as in the step kernels); writes
 * DEVICE float32 arrays out_u/out_v/out_w[n]; if out_var is non-NULL it also
 * receives the time-weighted corner variances, layout [3][n]. */
int mptrac_interp(mptrac_ctx* ctx, int64_t n, const double* lon, const double* lat,
                  const double* p, double t, float* out_u, float* out_v, float* out_w,
                  float* out_var, uintptr_t stream);

/* Raw Philox4x32-10 words: ctr is a DEVICE uint32 array [4][n] (counter word c
 * of item i at ctr[c*n + i]); out receives [4][n] words.  If normals is non-NULL
 * it receives the four Box-Muller normals [4][n] (float32) of each item. */
int mptrac_philox(const uint32_t* ctr, int64_t n, uint64_t seed, uint32_t* out,
                  float* normals, uintptr_t stream);

/* Read-only view of met slot `slot`: device pointer to its records
 * ([lat][lon][level] x 4 values: float32, or uint16 codes), its scales
 * (device float32 [4][nz]), its time and its record bytes.  Any output
 * pointer may be NULL. */
int mptrac_met_slot_info(const mptrac_ctx* ctx, int slot, const void** records,
                         const float** scales, double* t, size_t* bytes);

/* Number of CUDA kernels this library has launched in this process so far. */
uint64_t mptrac_kernel_launches(void);

/* Measurement aid, with no counterpart in the paper: one launch that copies
 * `bytes` bytes from DEVICE src to DEVICE dst `reps` times, loads and stores
 * cached in L2 only (not L1), each repetition with another thread-to-element
 * mapping.  With src and dst resident in L2 together (2 * bytes well below
 * the L2 size) it measures the L2 bandwidth that the gather roofline divides
 * by; with buffers far larger than L2, the DRAM copy bandwidth.  bytes must be
 * a multiple of 16 and both pointers 16-byte aligned (E_INVALID_ARG
 * otherwise); reps >= 1.  Asynchronous on `stream`. */
int mptrac_copy_probe(const void* src, void* dst, size_t bytes, int reps, uintptr_t stream);

/* Copies met slot `slot` into caller-owned DEVICE buffers: records_out
 * (mptrac_met_slot_info's `bytes` bytes) and scales_out (4*nz float32), on
 * `stream`.  Either output may be NULL. */
int mptrac_met_slot_copy(const mptrac_ctx* ctx, int slot, void* records_out, float* scales_out,
                         uintptr_t stream);

#ifdef __cplusplus
}
#endif
#endif /* MPTRAC_H */
