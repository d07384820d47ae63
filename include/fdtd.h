/*
 * fdtd.h -- C ABI of the GB300 FDTD + CPML library (libfdtd.so).
 *
 * The library advances the first-order acoustic pressure-velocity system
 *     p_t = -K div v,   v_t = -(1/rho) grad p          (paper Sec. 3.1)
 * with centred radius-4 (eighth-order) derivatives and a leapfrog step
 * (velocity half step from p^n, then pressure step from v^{n+1/2}), and the
 * convolutional PML of Sec. 3.2 in the six boundary slabs: inside the slab of
 * axis d every derivative delta_d f becomes (1/kappa_d) delta_d f + psi_d with
 * psi_d <- b_d psi_d + a_d delta_d f.  Source injection and receiver sampling
 * run inside the same kernel.  A discrete adjoint (the exact transpose of the
 * step) gives misfit gradients with respect to the velocity model and to the
 * CPML coefficient profiles.
 *
 * Conventions used by every entry point
 * -------------------------------------
 *  - Arrays are C order [nz][ny][nx] (x fastest) unless stated; "dev" means a
 *    CUDA device pointer, "host" a host pointer.
 *  - Spatial indices are 0-based (z, y, x) triples.
 *  - Faces are ordered -x, +x, -y, +y, -z, +z; CPML cells lie inside the grid.
 *  - Every call returns an fdtd_status; nothing throws or aborts across the
 *    ABI.  After a failure fdtd_last_error() holds a one-line reason.
 *  - Work is enqueued on the stream given in fdtd_desc and calls may return
 *    before it completes; calls that return host values (fdtd_set_model,
 *    fdtd_sync, fdtd_energy, fdtd_misfit) synchronise that stream.  Errors
 *    raised on the device (a bounded wait that gave up, non-finite values)
 *    are reported by the next synchronising call.
 *  - Ownership: the caller allocates all device memory.  fdtd_workspace_bytes
 *    sizes one workspace that the caller passes to fdtd_create and keeps alive
 *    until fdtd_destroy; the library carves every field, memory variable,
 *    table and checkpoint out of it and never allocates device memory.  The
 *    traces buffer given to fdtd_record is written in place and must outlive
 *    the steps that record into it.  Host arrays are copied before the call
 *    returns.
 *  - One context per host thread at a time.
 */
#ifndef FDTD_H
#define FDTD_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FDTD_ABI_VERSION 2

typedef struct fdtd_ctx fdtd_ctx;

typedef enum {
    FDTD_OK = 0,
    FDTD_EINVAL = 1,       /* an argument is out of range or inconsistent */
    FDTD_ENOMEM = 2,       /* workspace too small, or host allocation failed */
    FDTD_ECUDA = 3,        /* a CUDA runtime call or kernel launch failed */
    FDTD_ESTATE = 4,       /* call out of order (e.g. step before set_model) */
    FDTD_EUNSTABLE = 5,    /* c_max dt / h above the scheme's stability limit */
    FDTD_EDIVERGED = 6,    /* non-finite values detected */
    FDTD_ETIMEOUT = 7,     /* a bounded device-side wait gave up */
    FDTD_EUNSUPPORTED = 8  /* valid request the library does not provide */
} fdtd_status;

typedef enum {
    FDTD_F32 = 0,          /* p, v, psi stored in FP32 */
    FDTD_F16 = 1,          /* stored in FP16, arithmetic in FP32 registers */
    FDTD_BF16 = 2          /* stored in BF16, arithmetic in FP32 registers */
} fdtd_storage;

/* Field selectors for fdtd_get_field / fdtd_set_field.  Velocities and memory
 * variables are always exchanged in physical units, whatever the storage. */
typedef enum {
    FDTD_P = 0, FDTD_VX = 1, FDTD_VY = 2, FDTD_VZ = 3,
    FDTD_PSIV_X = 4, FDTD_PSIV_Y = 5, FDTD_PSIV_Z = 6,   /* memory of delta_d p   */
    FDTD_PSIP_X = 7, FDTD_PSIP_Y = 8, FDTD_PSIP_Z = 9,   /* memory of delta_d v_d */
    FDTD_ADJ_P = 10, FDTD_ADJ_VX = 11, FDTD_ADJ_VY = 12, FDTD_ADJ_VZ = 13,
    FDTD_ADJ_PSIV_X = 14, FDTD_ADJ_PSIV_Y = 15, FDTD_ADJ_PSIV_Z = 16,
    FDTD_ADJ_PSIP_X = 17, FDTD_ADJ_PSIP_Y = 18, FDTD_ADJ_PSIP_Z = 19
} fdtd_field;

typedef struct {
    int nx, ny, nz;          /* grid nodes; CPML cells included */
    int nshots;              /* independent wavefields sharing one model (>= 1) */
    double h;                /* grid spacing [m], equal on all axes */
    double dt;               /* time step [s] */
    int cpml_cells[6];       /* CPML cells per face (-x,+x,-y,+y,-z,+z), 0 = none */
    int storage;             /* fdtd_storage */
    int tblock_k;            /* time steps per block: 1, 2 or 4 (see fdtd_step_n) */
    int nt_max;              /* capacity of wavelet and trace buffers (steps) */
    int nrec_max;            /* receiver capacity */
    int checkpoint_every;    /* > 0: keep checkpoints every C steps (adjoint) */
    int cpml_grad;           /* != 0: also keep what dJ/d(CPML profile) needs */
    int cpml_local;          /* != 0: reserve per-node CPML coefficients (fdtd_set_cpml_local) */
    void *stream;            /* cudaStream_t to enqueue on; NULL = default */
} fdtd_desc;

/* ABI version of the loaded library (FDTD_ABI_VERSION). */
int fdtd_abi_version(void);

/* Short name of a status code; never NULL. */
const char *fdtd_status_string(int status);

/* Bytes of device workspace that fdtd_create needs for `desc` (host-only
 * computation; no CUDA call).  EINVAL if desc is invalid: a dimension < 1,
 * h or dt <= 0, 2 * cells > n on an axis, storage unknown, tblock_k not 1, 2 or 4,
 * nt_max < 1, nshots outside [1, 1024], nrec_max < 0, checkpoint_every < 0,
 * or cpml_grad set without checkpoint_every. */
int fdtd_workspace_bytes(const fdtd_desc *desc, size_t *bytes);

/* Create a context on the current CUDA device.  `workspace` (dev, 256-byte
 * aligned, >= fdtd_workspace_bytes) stays owned by the caller and must
 * outlive the context.  All fields start at zero, time index 0.  With the
 * environment variable FDTD_FAULT=alloc the call fails with ENOMEM before
 * touching the GPU (host-side failure injection for tests). */
int fdtd_create(const fdtd_desc *desc, void *workspace, size_t workspace_bytes,
                fdtd_ctx **out);

/* Release the context (host memory only; the workspace stays the caller's). */
int fdtd_destroy(fdtd_ctx *ctx);

/* One-line description of the last failure on this context ("" if none). */
const char *fdtd_last_error(const fdtd_ctx *ctx);

/* Velocity model (paper Sec. 3.1: p_t = -K div v, v_t = -(1/rho) grad p,
 * K = rho c^2).  vel_dev: float [nz][ny][nx] in m/s; rho_dev: NULL (density 1
 * everywhere) or float [nz][ny][nx], the density per node, collocated with p
 * and v (the velocity update at a node uses dt / rho of that node).  Both are
 * read during the call.  With a density the step and its adjoint read one
 * more table (4 B per node, shared by the shots); the adjoint's gradient is
 * then dJ/dc at fixed density.  Synchronises; EINVAL if a velocity or
 * density is not finite and positive; EUNSTABLE if max(c) dt / h exceeds the
 * collocated radius-4 leapfrog limit 2 / (sqrt(3) max_theta 2 sum_l a_l sin(l theta)) = 0.6672. */
int fdtd_set_model(fdtd_ctx *ctx, const float *vel_dev, const float *rho_dev);

/* Velocity scale of 16-bit storage: the stored velocity is scale * v (an
 * impedance scaling that keeps the stored v of the order of p; the memory
 * variables of the pressure update carry the same scale).  scale = 0 (the
 * default) takes the model's maximum velocity.  Takes effect at the next
 * fdtd_set_model; FP32 storage ignores it.  Contexts that hold parts of one
 * grid (fdtd_exchange) must store at the same scale.  EINVAL for a negative
 * or non-finite scale. */
int fdtd_set_velocity_scale(fdtd_ctx *ctx, double scale);

/* CPML grading of Sec. 3.2 / Tab. 2 on the cells given at create time:
 *   sigma = sigma_max rho^q, sigma_max = -(q+1) c_ref ln(R) / (2 L h),
 *   kappa = 1 + (kappa_max - 1) rho^q, alpha = alpha_frac sigma_max (1 - rho),
 *   b = exp(-(sigma/kappa + alpha) dt), a = sigma (b - 1) / (kappa (sigma + kappa alpha)),
 * with normalised depth rho = (L - j)/L at cell j (j = 0 outermost).
 * c_ref <= 0 selects the model's maximum velocity (requires fdtd_set_model).
 * Coefficients are computed on the host in double and stored as float.
 * EINVAL for R outside (0, 1], kappa_max < 1, alpha_frac < 0 or q < 0. */
int fdtd_set_cpml(fdtd_ctx *ctx, double R, double kappa_max, double alpha_frac,
                  int q, double c_ref);

/* Local-velocity CPML grading (heterogeneous media, the extension Sec. 7
 * names): at every node of the d-slab, sigma_max takes the velocity of that
 * node in place of one reference velocity,
 *   sigma_max(c) = -(q+1) c ln(R) / (2 L h),  sigma = sigma_max rho^q,
 *   alpha = alpha_frac sigma_max(c) (1 - rho),  kappa = 1 + (kappa_max - 1) rho^q,
 * with the node's normalised depth rho along d and the face's own L, so the
 * continuous round trip is R for every column.  b, a are computed per slab
 * node on the device in double and stored as float (8 B per slab node and
 * axis, shared by the shots, read by every step); 1/kappa stays per axis.
 * vel_dev: float [nz][ny][nx] in m/s, read during the call (normally the
 * model given to fdtd_set_model).  Requires cpml_local at create time
 * (ESTATE otherwise) and fdtd_set_model first (ESTATE).  Replaces any
 * previous grading; fdtd_set_cpml or fdtd_set_cpml_ska replace it in turn.
 * EINVAL for parameters as in fdtd_set_cpml or a slab velocity that is not
 * finite and positive; EUNSUPPORTED with 16-bit storage or the staggered
 * form.  fdtd_adjoint_step_n transposes the per-node coefficients (its dJ/dc
 * holds them fixed); the CPML-profile gradient, which is per axis and node
 * index, is not provided with them (grad_cpml: EUNSUPPORTED).  Synchronises. */
int fdtd_set_cpml_local(fdtd_ctx *ctx, const float *vel_dev, double R, double kappa_max,
                        double alpha_frac, int q);

/* Elliptic anisotropy (the acoustic system of the paper's 2D CPML
 * demonstration, Sec. 5): the pressure update becomes
 *   p <- p - dt K sum_d kr_d [ (1/kappa_d) delta_d v_d + psi_{p,d} ],
 * so the wave speed along axis d is c sqrt(kr_d).  kr (host double[3],
 * x, y, z) must be finite and positive; (1, 1, 1) is the isotropic default.
 * The stability limit becomes c_max dt / h <= 2 / (sqrt(sum_d kr_d) max_theta
 * 2 sum_l a_l sin(l theta)); EUNSTABLE (factors unchanged) if a set model
 * violates it, and fdtd_set_model checks it too.  The CPML grading keeps
 * its single c_ref.  fdtd_adjoint_step_n transposes the anisotropic step
 * (axis d's bracket keeps its factor kr_d, also through the CPML memory
 * variables); its gradients are with respect to the base modulus K = c^2.
 * A 2D run is ny = 1 with no y layer (the zero values beyond the grid make
 * delta_y vanish there). */
int fdtd_set_anisotropy(fdtd_ctx *ctx, const double kr[3]);

/* Staggered (Yee) form of the same system (Sec. 3.1 names both grids):
 * on = 1 keeps p at the nodes and v_d[i] at the half node i + 1/2 along d,
 * with the staggered radius-4 derivatives
 *   v_d <- v_d - dt/rho [ (1/kappa) D+ p + psi_v ],  D+ f[i] = (1/h) sum_l c_l (f[i+l] - f[i+1-l]),
 *   p   <- p - dt K sum_d kr_d [ (1/kappa) D- v_d + psi_p ],  D- f[i] = (1/h) sum_l c_l (f[i+l-1] - f[i-l]),
 * c = (1225/1024, -245/3072, 49/5120, -5/7168), zero values beyond the grid
 * (so D- = -D+^T).  The velocity memory variables keep the slab index set
 * of p and the grading of fdtd_set_cpml at the half-node depth
 * (lo - i - 1/2)/lo on a low face and min(1, (i + 1/2 - (n - 1 - hi))/hi) on
 * a high face.  Every array keeps its layout; FDTD_VX etc. then hold the
 * half-node values.  The stability limit becomes
 * 2 / (sqrt(sum_d kr_d) 2 sum_l |c_l|) = 0.44884 for kr = 1.
 * on = 0 restores the collocated default.  Chosen before the first step
 * (ESTATE after it until fdtd_reset).  EUNSUPPORTED for 16-bit storage, with
 * a density, with learned profiles (fdtd_set_cpml_ska) or with the local
 * grading.  fdtd_adjoint_step_n transposes the staggered step (D+^T = -D-,
 * D-^T = -D+, half-node velocity profiles); the CPML-profile gradient is not
 * provided for it (grad_cpml: EUNSUPPORTED).  EUNSTABLE (form unchanged) if
 * a set model violates the limit; fdtd_set_model checks it. */
int fdtd_set_staggered(fdtd_ctx *ctx, int on);

/* Per-cell (sigma, kappa, alpha) for a layer of L equal cells on every face
 * (all six cpml_cells equal to L): ska_dev float [L][3], cell j = 0
 * outermost.  Converted to (b, a, 1/kappa) on the device.  Used by the
 * learned CPML.  EINVAL if the faces differ. */
int fdtd_set_cpml_ska(fdtd_ctx *ctx, const float *ska_dev);

/* Source per shot: src_zyx (host int [nshots][3]) and wavelet_dev (dev float
 * [nshots][nt], copied).  After the pressure update of step n, w[shot][n] is
 * added to p at the source node (additive pressure source; samples n >= nt
 * add nothing).  The paper gives only the source's time function, the Ricker
 * pulse of Sec. 4.2 (the caller samples it, w[n] = s(n dt)); how it enters the
 * update is left open, and this additive injection after the pressure step,
 * with the amplitude as given, is the reading taken here and by the oracle.  EINVAL if a node is outside the grid or nt > nt_max. */
int fdtd_inject(fdtd_ctx *ctx, const int *src_zyx, const float *wavelet_dev, int nt);

/* Receivers, shared by all shots: rec_zyx (host int [nrec][3]).  After the
 * source of step n, traces_dev[shot][n][r] = p at receiver r for every
 * n < nt_max (the paper samples no receivers; its Sec. 4.2 reflection ratios
 * compare the pressure at fixed nodes, and sampling p^{n+1} after the source
 * of step n is the reading taken here and by the oracle) (traces_dev: dev float [nshots][nt_max][nrec], written in
 * place).  nrec = 0 disables recording.  EINVAL if a node is outside the
 * grid or nrec > nrec_max. */
int fdtd_record(fdtd_ctx *ctx, const int *rec_zyx, int nrec, float *traces_dev);

/* Advance every shot by n full time steps (one fused kernel per step).
 * With checkpoint_every = C > 0 the state is saved before every step whose
 * index is a multiple of C (up to nt_max).  ESTATE before set_model /
 * set_cpml; EINVAL if n < 0.
 *
 * Temporal blocking, tblock_k = k in {2, 4} (the enlarged-ghost idea of
 * paper Sec. 3.3, g = 2 r s, applied to z bands of one device): whole
 * blocks of k steps cut the z range into bands of >= 8 planes (96 by
 * default, environment variable FDTD_TBAND), each launched in chunks of at
 * most 32 planes (96 with 16-bit storage; FDTD_TBCHUNK); step s of a block
 * runs on a band as soon as step s - 1 has finished that band and its two
 * neighbours, so the k steps' launches overlap.  The library enqueues on k
 * internal streams that join `stream` before the call returns (events; no
 * host wait).  Results are identical to
 * k = 1, node for node.  Steps left over after the whole blocks, and any
 * block with a checkpoint inside it, run as single steps. */
int fdtd_step_n(fdtd_ctx *ctx, int n);

/* Discrete adjoint of the last n = current-time steps (run backwards from the
 * current time index to 0 from the checkpoints, recomputing each segment):
 * the exact transpose of the forward step.  resid_dev (dev float
 * [nshots][nt_max][nrec], the misfit derivative dJ/dtrace) is injected at the
 * receivers.  grad_vel_dev (dev float [nz][ny][nx]) receives += dJ/dc summed
 * over shots (K = rho c^2, dJ/dc = 2 rho c dJ/dK; density, anisotropy and CPML
 * coefficients held fixed).  grad_cpml_dev
 * (dev float [3][3][nmax], nullable; nmax = max(nx, ny, nz); [axis x,y,z]
 * [b, a, 1/kappa][node]) receives += dJ/d(profile) and needs cpml_grad at
 * create time (EINVAL otherwise).  Needs FP32 storage,
 * checkpoint_every > 0 and n equal to the current time index (ESTATE
 * otherwise).  grad_cpml is for the collocated form with the 1D grading
 * (EUNSUPPORTED with the staggered form or fdtd_set_cpml_local).  Leaves the
 * forward state undefined (call fdtd_reset). */
int fdtd_adjoint_step_n(fdtd_ctx *ctx, int n, const float *resid_dev,
                        float *grad_vel_dev, float *grad_cpml_dev);

/* Copy one field of one shot to/from a dense float [nz][ny][nx] device array
 * in physical units.  Memory variables are full-volume arrays that are zero
 * outside their slab (values outside the slab are ignored on set). */
int fdtd_get_field(fdtd_ctx *ctx, int which, int shot, float *dst_dev);
int fdtd_set_field(fdtd_ctx *ctx, int which, int shot, const float *src_dev);

/* Halo exchange of the domain decomposition of Sec. 3.3: copy the stepped
 * state -- p, v and the CPML memory variables, every shot -- over the box
 * box = {z0, z1, y0, y1, x0, x1} of dst's grid from the nodes
 * (z + shift[0], y + shift[1], x + shift[2]) of src's grid.  The two contexts
 * hold parts of one grid (with the CPML on the grid's outer faces only, as in
 * Sec. 3.3), so a memory variable psi_d is copied where both keep it (a node
 * in the d-slabs of both).  Both must have the same storage, shots and form
 * and the same time index (ESTATE otherwise); EINVAL if a box leaves either
 * grid, or if the two store velocities at different scales (see
 * fdtd_set_velocity_scale).  The copy is one kernel on dst's stream that
 * reads src's arrays directly: src's last step must be complete or on the
 * same stream.  The adjoint state and checkpoints are not exchanged.  Both
 * contexts must live on the same GPU (EUNSUPPORTED otherwise: parts on
 * several GPUs would need peer access, which the library does not set up). */
int fdtd_exchange(fdtd_ctx *dst, const fdtd_ctx *src, const int box[6], const int shift[3]);

/* Zero every field and memory variable, time index 0 (model, CPML, source and
 * receivers are kept). */
int fdtd_reset(fdtd_ctx *ctx);

/* Current time index (steps taken since create/reset). */
int fdtd_time(const fdtd_ctx *ctx, int *t);

/* Divergence detection (off by default): after every `every` steps of
 * fdtd_step_n the library sums p^2 over every node of every shot in FP64 on
 * the device; a sum that is not finite, or above `limit` when limit > 0,
 * raises a device error that the next synchronising call (fdtd_sync)
 * reports as EDIVERGED.  No host synchronisation; one reduction over p per
 * check (4 B per node in FP32).  every = 0 turns it off.  EINVAL for
 * every < 0 or a NaN limit. */
int fdtd_set_divergence_check(fdtd_ctx *ctx, int every, double limit);

/* Set the time index (resume: with the fields restored by fdtd_set_field, a
 * run continues from step t, sampling wavelets and recording traces at t and
 * after).  EINVAL if t < 0; EUNSUPPORTED for a context with checkpoints,
 * whose adjoint replays from step 0. */
int fdtd_set_time(fdtd_ctx *ctx, int t);

/* Wait for the stream and report device-side errors (ETIMEOUT, EDIVERGED). */
int fdtd_sync(fdtd_ctx *ctx);

/* sum of p^2 over the box [z0,z1) x [y0,y1) x [x0,x1) of one shot, accumulated
 * in FP64 on the device; box = {z0, z1, y0, y1, x0, x1}.  Synchronises.
 * This is the "normalized field energy" of the paper's CPML demonstration
 * (Sec. 4.2, energy-decay figure), read as the sum of p^2 over a box, to be
 * normalised by its peak over time by the caller. */
int fdtd_energy(fdtd_ctx *ctx, int shot, const int box[6], double *out);

/* Data misfit J = 1/2 sum (traces - dobs)^2 over [nshots][nt][nrec] of the
 * recorded traces (first nt steps), accumulated in FP64 on the device.  The
 * paper has no inversion; this L2 misfit is the objective whose gradient
 * fdtd_adjoint_step_n computes (resid is its dJ/dtrace), and Sec. 4.1's
 * relative L2 error is the same norm;
 * resid_dev (nullable, dev float [nshots][nt_max][nrec]) receives
 * traces - dobs for n < nt and 0 beyond.  dobs_dev: dev float
 * [nshots][nt_max][nrec].  Synchronises. */
int fdtd_misfit(fdtd_ctx *ctx, const float *dobs_dev, int nt, float *resid_dev, double *out);

/* Kernel classes of fdtd_timing. */
typedef enum {
    FDTD_TIMING_STEP = 0,     /* the fused forward step kernel (also its recompute launches in the adjoint) */
    FDTD_TIMING_ADJOINT = 1   /* the adjoint step: the fused adjoint kernel (node-per-thread kernels with grad_cpml) */
} fdtd_timing_class;

/* Device-side timing of the library's kernels (the CUDA events per step of
 * the measurement plan; the paper times whole runs by wall clock, Sec. 5).
 * on != 0 records a CUDA event pair around every launch of each kernel class
 * on the stream it is launched on, and clears the totals; on = 0 stops
 * recording (totals are kept).  Events are created on the first call with
 * on != 0 and destroyed with the context.  Every 4096 launches of a class
 * the host waits for the launches recorded so far (a synchronisation), so
 * timing is meant for measurement runs. */
int fdtd_set_timing(fdtd_ctx *ctx, int on);

/* Milliseconds of device time and number of launches of one kernel class
 * (fdtd_timing_class) since timing was switched on: the sum over launches of
 * each launch's own start-to-end event interval.  Synchronises the stream
 * (and the temporal-blocking streams).  EINVAL for an unknown class. */
int fdtd_timing(fdtd_ctx *ctx, int kernel_class, double *ms, long long *launches);

/* Largest n accepted by fdtd_misfit_noalloc: 4096 partial sums of 65536 values. */
#define FDTD_NOALLOC_MISFIT_MAX 268435456LL

/* The data misfit of fdtd_misfit, J = 1/2 sum_i (traces[i] - dobs[i])^2 over
 * n floats accumulated in FP64, for callers that cannot allocate device
 * memory.  The paper has no counterpart to this entry point.  It needs no
 * context and allocates nothing, so it suits callers whose device memory
 * belongs to another allocator with a fixed budget (e.g. a framework's caching
 * allocator) or loops where cudaMalloc, which may synchronise the device, is
 * not allowed.  Its scratch is a 33 KB static device array that every GPU
 * loading the library keeps until the process exits.
 *   traces_dev, dobs_dev: dev float [n]; resid_dev: dev float [n] receiving
 *   traces - dobs, or NULL; out_host: host double receiving J; stream:
 *   cudaStream_t (NULL = default).  Synchronises the stream.
 *   EINVAL if a pointer is NULL or n is outside [1, FDTD_NOALLOC_MISFIT_MAX];
 *   ECUDA if a CUDA call fails.
 * Every call looks up the scratch array's device address on the current
 * device (a host-side query); the first call on a device also loads the
 * library's device code there, its set-up, so make that first call before any
 * stream capture begins on the device.  All calls on a device share the
 * scratch array, so calls that overlap on the GPU (e.g. on two streams at
 * once) race and must be serialised by the caller. */
int fdtd_misfit_noalloc(const float *traces_dev, const float *dobs_dev, long long n, float *resid_dev,
                        double *out_host, void *stream);

/* Per-cell (sigma, kappa, alpha) of the polynomial grading of Sec. 3.2 /
 * Tab. 2 for a layer of L cells (the formulas of fdtd_set_cpml, in double on
 * the host): ska_host double [L][3], cell j = 0 outermost at normalised depth
 * (L - j)/L.  The learned CPML's fallback and the target of its pre-fit; the
 * layout of fdtd_set_cpml_ska.  Needs no context and no GPU.  EINVAL for L
 * outside [1, 1024], h or c_ref <= 0, or parameters as in fdtd_set_cpml. */
int fdtd_cpml_grading(int L, double h, double c_ref, double R, double kappa_max, double alpha_frac,
                      int q, double *ska_host);

/* Chain rule of the learned CPML: from grad_cpml (layout of
 * fdtd_adjoint_step_n) and the per-cell ska_dev [L][3] given to
 * fdtd_set_cpml_ska, write gska_dev [L][3] = dJ/d(sigma, kappa, alpha). */
int fdtd_cpml_ska_backward(fdtd_ctx *ctx, const float *ska_dev, const float *grad_cpml_dev,
                           float *gska_dev);

/* ---- learned-CPML network (4 -> 64 -> 64 -> 3, tanh; no paper counterpart
 * beyond Sec. 7's future-work note; the CPML it feeds is Sec. 3.2) ----
 * theta: dev float [4675] = W1[64][4], b1[64], W2[64][64], b2[64], W3[3][64], b3[3].
 * X: dev float [n][4] features.  out: dev float [n][3] =
 *   (sigma_scale softplus(o0), 1 + softplus(o1), alpha_scale softplus(o2)).
 * act: dev float [n][131] saved activations (h1[64], h2[64], o[3]).
 * All three enqueue on `stream` (cudaStream_t, NULL = default); n <= 1024. */
int fdtd_mlp_forward(const float *theta, const float *X, int n, float sigma_scale,
                     float alpha_scale, float *out, float *act, void *stream);
/* gtheta (dev float [4675]) = dJ/dtheta from gout (dev float [n][3]). */
int fdtd_mlp_backward(const float *theta, const float *X, int n, const float *act,
                      const float *gout, float sigma_scale, float alpha_scale,
                      float *gtheta, void *stream);
/* Gradient of the learned grading's pre-fit loss (fitting the network to a
 * target grading, e.g. fdtd_cpml_grading's):
 *   loss = sum_j [((sigma_j - s*_j)/sigma_scale)^2 + (kappa_j - k*_j)^2 + ((alpha_j - a*_j)/alpha_scale)^2],
 * out, target: dev float [n][3] (sigma, kappa, alpha); gout: dev float [n][3]
 * = dloss/dout; loss: dev float [1] or NULL.  Summed in double; one block on
 * `stream`; n <= 1024. */
int fdtd_mlp_fit_gradient(const float *out, const float *target, int n, float sigma_scale,
                          float alpha_scale, float *gout, float *loss, void *stream);
/* Adam (Kingma & Ba) on nparam values; step t >= 1. */
int fdtd_adam_step(float *theta, const float *grad, float *m, float *v, int nparam, int t,
                   float lr, float beta1, float beta2, float eps, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* FDTD_H */
