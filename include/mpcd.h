/*
 * mpcd.h - C ABI of the GB300 (sm_103a) MPCD time step with rigid-body
 * discrete-particle colloids (Bush, Palmer, Howard, arXiv 2604.14307).
 *
 * One step of the method (Sec. II):
 *   stream    solvent ballistic drift with periodic wrap (Sec. II.A) and one
 *             velocity-Verlet step of the rigid bodies with the Miller et al.
 *             quaternion integrator and core-shifted WCA forces (Eq. 1);
 *   couple    PRE:  surface-site positions from each body's pose and
 *                   thermalisation of the site velocities (Eq. 7, Sec. II.B.2);
 *             POST: transfer of the sites' momentum change to the body
 *                   (Eqs. 3-4) and reset of the sites to rigid motion (Eq. 5);
 *   collide   random grid shift, cell binning, per-cell mass/momentum/energy
 *             sums, SRD rotation (or MPCD-AT) with the cell-level thermostat
 *             (Sec. II.A).
 * mpcd_step() runs whole steps; it is equivalent to calling, per step,
 * stream, couple(PRE), collide, couple(POST) in that order.
 *
 * Conventions
 *   - Every call returns an mpcd_status; nothing throws across the ABI.
 *   - The library owns all device memory of a context (through the optional
 *     allocator).  Host buffers belong to the caller; they are only read or
 *     written during the call that receives them.
 *   - `stream` arguments are cudaStream_t values passed as void* (NULL is the
 *     legacy default stream).  Calls enqueue asynchronously on that stream
 *     unless their comment says they synchronise.  Errors are sticky: after a
 *     failure every further call on the context returns the same status until
 *     mpcd_destroy(); mpcd_last_error() describes it.
 *   - A context is used by one host thread at a time.
 *   - Lengths are in units of the cell size a = 1; periodic boxes have integer
 *     edges L (cells per edge) and positions lie in [0, L).  Quaternions are
 *     (w, x, y, z), unit norm, body -> space.  Angular momenta are space-frame.
 */
#ifndef MPCD_H
#define MPCD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mpcd_ctx mpcd_ctx;

typedef enum {
    MPCD_OK = 0,
    MPCD_ERR_ARG = -1,      /* invalid argument or size; nothing was changed */
    MPCD_ERR_CUDA = -2,     /* a CUDA runtime call failed (sticky) */
    MPCD_ERR_OOM = -3,      /* device allocation failed */
    MPCD_ERR_TIMEOUT = -4,  /* a bounded device wait gave up (sticky) */
    MPCD_ERR_STATE = -5     /* the device detected an invalid state, e.g. a
                               particle moved more than one box length in a
                               step or a cell exceeded 65535 particles */
} mpcd_status;

enum { MPCD_P64 = 0,   /* FP64 solvent state, FP64 cell sums (plain form) */
       MPCD_P32 = 1 }; /* FP32 solvent state, int64 fixed-point cell sums,
                          FP64 bodies */
enum { MPCD_SRD = 0,   /* stochastic rotation by alpha about a random axis */
       MPCD_AT = 1 };  /* Andersen-thermostat collision (MPCD-AT) */
enum { MPCD_PRE = 0, MPCD_POST = 1 };

/* Physical and numerical parameters (Sec. II.A, Sec. III). */
typedef struct {
    double kT;            /* temperature of the thermostat and of Eq. 7 */
    double dt;            /* streaming interval = MD step = collision period */
    double alpha_deg;     /* SRD rotation angle (130 in the paper) */
    double m_solvent;     /* solvent particle mass */
    int32_t rule;         /* MPCD_SRD or MPCD_AT */
    int32_t thermostat;   /* cell-level thermostat for SRD (AT is intrinsically
                             thermostatted and ignores it): each cell's relative
                             kinetic energy is rescaled to E' ~ Gamma(3(N_c-1)/2, kT)
                             (Eq. 6).  0: off; 1: E' drawn without rejection as a
                             sum of unit exponentials (the reference form);
                             2: E' drawn by the rejection method of Marsaglia and
                             Tsang (same distribution, about one Philox block per
                             cell; FP32 and FP64 may decide a rejection differently
                             in rare cells) */
    int32_t precision;    /* MPCD_P64 or MPCD_P32 */
    int32_t naive_transfer; /* 1: skip Eq. 7 (negative control of Fig. S1) */
    uint64_t seed;        /* Philox4x32-10 key */
    int32_t sort_period;  /* steps between spatial re-sorts of the solvent;
                             0 = default (20), < 0 = never */
    int32_t angular;      /* 1: angular-momentum-conserving variant of the rule
                             (SRD+a, MPCD-AT+a, the modification Sec. II.A cites):
                             after the rule every cell with >= 2 members gets the
                             rigid rotation v' = v* + w x r_c that restores its
                             angular momentum about its centre of mass (r_c on the
                             2^-20 lattice of the binning rule; least-norm w for
                             collinear members).  Colloid sites take part like
                             solvent; their corrected velocities enter the
                             transfer to the body.  Needs one site mass for all
                             shapes (MPCD_ERR_ARG otherwise); steps run unfused.
                             0: off */
} mpcd_params;

/* A rigid discrete-particle template in its principal-axis frame with its
 * site centre of mass at the origin (Sec. II.B).  All arrays are copied. */
typedef struct {
    int32_t n_sites;
    const double *b;        /* [n_sites][3] body-frame site offsets */
    const double *m;        /* [n_sites] site masses (> 0) */
    int32_t n_centres;
    const double *centres;  /* [n_centres][3] massless WCA centres (Eq. 1) */
    double wca_d;           /* centre diameter d; Delta = d - sigma, sigma = 1 */
} mpcd_shape_desc;

/* One independent periodic box; replicas are simulated together. */
typedef struct {
    int32_t L[3];             /* cells per edge (3 to 2047 each: the binning rule forms
                                 floor(x 2^20) in 32 bits) */
    int64_t n_solvent;        /* solvent particles of this replica */
    int32_t n_bodies;
    int32_t stream_id;        /* >= 0, distinct within a context: the replica's random
                                 streams use the Philox key (seed_lo, seed_hi ^ stream_id).
                                 Give each replica its index in the whole ensemble and
                                 its trajectory does not depend on how the ensemble is
                                 split over contexts or GPUs. */
    const int32_t *body_shape;  /* [n_bodies] shape index (copied) */
} mpcd_replica_desc;

/* Optional device allocator (e.g. a framework's caching allocator).  Both
 * functions are called on the creating thread; alloc returns NULL on failure
 * and otherwise device memory aligned to at least 16 bytes (the kernels' bulk
 * copies require it; cudaMalloc and PyTorch's caching allocator give 256 and
 * 512). */
typedef struct {
    void *(*alloc)(size_t bytes, void *user);
    void (*free)(void *ptr, void *user);
    void *user;
} mpcd_allocator;

/* Host-side state, all replicas concatenated in replica order.  Solvent rows
 * are in tag order (the order given to mpcd_set_state). */
typedef struct {
    void *x;        /* [N_s][3] positions: float for MPCD_P32, double for P64 */
    void *v;        /* [N_s][3] velocities, same type */
    double *R;      /* [B][3] body centres of mass (site COM) */
    double *q;      /* [B][4] orientations */
    double *P;      /* [B][3] linear momenta (Eq. 3) */
    double *Lm;     /* [B][3] space-frame angular momenta (Eq. 4) */
    int64_t step;   /* completed steps; keys the random streams */
} mpcd_host_state;

typedef struct {
    int64_t n_solvent, n_bodies, n_sites, n_cells;
    int32_t n_replicas, n_shapes;
    int64_t device_bytes;     /* bytes the context holds on the device */
    int32_t sum_words;        /* words per cell of the debug sums (see below) */
    int32_t param_bytes;      /* bytes per cell of the debug parameters */
} mpcd_sizes_t;

/* Global diagnostics in FP64 (computed on the device). */
typedef struct {
    double p_solvent[3];      /* sum m v over the solvent */
    double p_bodies[3];       /* sum P over the bodies */
    double ke_solvent;        /* sum m v^2 / 2 over the solvent */
    double ke_trans;          /* sum |P|^2 / 2M over the bodies */
    double ke_rot;            /* sum w.I.w / 2 over the bodies */
    int64_t step;
} mpcd_diag;

/* Create a context on CUDA device `device`.  Validates every argument
 * (MPCD_ERR_ARG), builds the per-shape mass and principal moments, allocates
 * the device state (MPCD_ERR_OOM) and zeroes it; call mpcd_set_state next.
 * The paper's cell size a = 1 is the only one supported.  A replica with more
 * than one body needs every box edge above twice the largest WCA cutoff
 * (d_ij - sigma + 2^(1/6) sigma, Eq. 1) so that each centre pair has one
 * minimum image; the P32 form needs one site mass for all shapes. */
int mpcd_create(const mpcd_params *params, int32_t n_shapes, const mpcd_shape_desc *shapes,
                int32_t n_replicas, const mpcd_replica_desc *replicas,
                const mpcd_allocator *allocator, int32_t device, mpcd_ctx **out);

/* Release every resource of the context.  NULL-safe.  Synchronises. */
int mpcd_destroy(mpcd_ctx *ctx);

/* Upload a full state from host buffers (pinned or pageable) and compute the
 * initial WCA forces.  Positions must lie in [0, L). */
int mpcd_set_state(mpcd_ctx *ctx, const mpcd_host_state *state, void *stream);

/* Download the full state into caller buffers sized by mpcd_sizes().
 * Solvent rows come back in tag order.  Synchronises the stream. */
int mpcd_get_state(mpcd_ctx *ctx, mpcd_host_state *state, void *stream);

/* a1 + a9: stream the solvent and advance the bodies by one MD step. */
int mpcd_stream(mpcd_ctx *ctx, void *stream);

/* MPCD_PRE (a3, a4): site poses and Eq. 7 thermalisation, sites binned into
 * the cell sums; MPCD_POST (a8): site collision, momentum transfer to the
 * bodies, step counter advanced.  PRE must precede mpcd_collide and POST
 * follow it. */
int mpcd_couple(mpcd_ctx *ctx, int32_t phase, void *stream);

/* a2, a5-a7: grid shift, solvent binning, cell sums, collision parameters,
 * solvent collision. */
int mpcd_collide(mpcd_ctx *ctx, void *stream);

/* Run `nsteps` whole steps (>= 0).  Steps are software-pipelined: the
 * solvent pass of step n also streams and bins for step n+1, so the solvent
 * arrays are read and written once per step.  Results are identical to the
 * unpipelined sequence. */
int mpcd_step(mpcd_ctx *ctx, int64_t nsteps, void *stream);

/* Re-sort the solvent storage by cell for memory locality.  canonical != 0
 * orders each cell by tag, making the storage order deterministic.  Does not
 * change any result. */
int mpcd_sort(mpcd_ctx *ctx, int32_t canonical, void *stream);

/* ------------------------------------------------------------------------
 * Spatial domain decomposition of one box into slabs along z (Sec. II.A).
 *
 * One context per slab [z_lo, z_hi) of a single periodic box (e.g. one GPU
 * each).  The context holds the box's whole cell grid, a subset of its solvent
 * (every particle keeps its box-wide id, the counter of its random draws) and
 * all of its bodies (the bodies are replicated: every slab integrates them
 * alike).  A slab bins and transfers only the surface sites whose z lies in
 * its range.  Under the random grid shift the shifted cell layer that straddles
 * a slab face holds particles of both neighbours; their partial cell words are
 * exact integers (P32), so adding the neighbour's partial words of the two
 * layers next to each face, z_face - 1 and z_face, gives the words of the whole
 * box bit for bit.  One step of a slab, in order:
 *   mpcd_stream                        solvent and bodies move
 *   mpcd_slab_extract, _export         particles now outside [z_lo, z_hi) leave
 *   mpcd_slab_insert                   the neighbours' leavers arrive
 *   mpcd_couple(MPCD_PRE)              sites; only the slab's own are binned
 *   mpcd_collide_begin                 solvent binned into partial words
 *   mpcd_layer_words (get, then add)   the face layers' words completed
 *   mpcd_collide_end                   cell parameters and the collision
 *   mpcd_couple_post_partial           the slab's share of each body's transfer
 *   mpcd_apply_impulse                 the sum over all slabs applied; step done
 * (paper_2604_14307_gb300/domain.py drives it over torch.distributed.)  The
 * angular-momentum-conserving variant is not supported here (MPCD_ERR_ARG).
 * ------------------------------------------------------------------------ */

/* A slab context: box edges L (cells), the box's total solvent count (the base
 * of the sites' random-stream ids), room for `capacity` solvent particles
 * (<= n_solvent_total), all n_bodies bodies (shape indices copied), owned
 * range [z_lo, z_hi) with 0 <= z_lo < z_hi <= L[2] and at least 2 cells unless
 * it is the whole box.  The solvent is empty until mpcd_slab_set_state. */
int mpcd_create_slab(const mpcd_params *params, int32_t n_shapes, const mpcd_shape_desc *shapes,
                     const int32_t L[3], int64_t n_solvent_total, int64_t capacity, int32_t n_bodies,
                     const int32_t *body_shape, int32_t z_lo, int32_t z_hi, const mpcd_allocator *allocator,
                     int32_t device, mpcd_ctx **out);

/* Load a slab: n solvent particles with box-wide ids tags[n] (uint32), host
 * rows x[n][3], v[n][3] (float for P32, double for P64) inside the box, and
 * every body's R[B][3], q[B][4], P[B][3], Lm[B][3]; step keys the random
 * streams.  Synchronises.  (mpcd_set_state / mpcd_get_state refuse a slab.) */
int mpcd_slab_set_state(mpcd_ctx *ctx, int64_t n, const uint32_t *tags, const void *x, const void *v,
                        const double *R, const double *q, const double *P, const double *Lm, int64_t step,
                        void *stream);
/* The slab's state: *n its solvent count; with non-NULL buffers its particles
 * (ids, x, v in storage order) and every body.  Synchronises. */
int mpcd_slab_get_state(mpcd_ctx *ctx, int64_t *n, uint32_t *tags, void *x, void *v, double *R, double *q,
                        double *P, double *Lm, void *stream);
/* Move the particles whose z is outside [z_lo, z_hi) out of the slab (storage
 * order kept for both groups); *n_left their number.  mpcd_slab_export copies
 * them (ids, x[n][3], v[n][3]) to host buffers.  Synchronise. */
int mpcd_slab_extract(mpcd_ctx *ctx, int64_t *n_left, void *stream);
int mpcd_slab_export(mpcd_ctx *ctx, uint32_t *tags, void *x, void *v, void *stream);
/* Append n particles (ids, x, v; inside the box) after the slab's own;
 * MPCD_ERR_ARG beyond the capacity.  Synchronises. */
int mpcd_slab_insert(mpcd_ctx *ctx, int64_t n, const uint32_t *tags, const void *x, const void *v, void *stream);

/* mpcd_collide in two halves (no exchange protocol, not the +a variant):
 * _begin bins the solvent into the cell words at the current step's grid
 * shift; _end turns the words into collision parameters and collides. */
int mpcd_collide_begin(mpcd_ctx *ctx, void *stream);
int mpcd_collide_end(mpcd_ctx *ctx, void *stream);

/* The cell words of the z-layers [layer0, layer0 + n_layers) of the shifted
 * grid (a context with one replica; layer0 + n_layers <= L[2]): add = 0 copies
 * them to words[sum_words][n_layers L[0] L[1]] (the layout of mpcd_debug_cells,
 * int64 for P32, double for P64), add = 1 adds that array to them.
 * Synchronises. */
int mpcd_layer_words(mpcd_ctx *ctx, int32_t layer0, int32_t n_layers, void *words, int32_t add, void *stream);

/* The POST coupling in two halves: _partial runs the sites' collision and
 * returns, without applying it, each body's momentum and angular-momentum
 * change from this context's (for a slab: its own) sites, dPL[B][6] in FP64
 * (Eqs. 3-4; synchronises); mpcd_apply_impulse adds dPL[B][6] to the bodies and
 * ends the step (the step counter advances). */
int mpcd_couple_post_partial(mpcd_ctx *ctx, double *dPL, void *stream);
int mpcd_apply_impulse(mpcd_ctx *ctx, const double *dPL, void *stream);

/* Binning as a counting sort (Sec. II.A; the cell assignment under the random
 * grid shift): the canonical member order of the collision at the current
 * step.  Call it between mpcd_couple(PRE) and mpcd_collide (for a context
 * without colloids, any time after mpcd_stream): every solvent particle at its
 * current position under the grid shift of that collision, and every site in
 * the cell its PRE coupling assigned, is counted into its cell (histogram), the
 * counts are scanned into each cell's first slot, the members are scattered and
 * each cell's members are ordered solvent before sites, each by ascending id.
 *   order       host int64[n_solvent + n_sites]: the members cell by cell; a
 *               solvent particle is given as its row in the host state arrays
 *               (replica offset + tag), a site as n_solvent + its index in the
 *               body-major site order
 *   cell_start  host int64[n_cells + 1]: cell c holds order[cell_start[c] ..
 *               cell_start[c + 1]), cells numbered replica by replica
 * The result is unique (integer work), so it is reproducible bit for bit.  The
 * time step itself never needs it: its cell sums are order-independent integer
 * sums.  Scratch is allocated on the first call.  Changes no state;
 * synchronises the stream. */
int mpcd_cell_order(mpcd_ctx *ctx, int64_t *order, int64_t *cell_start, void *stream);

/* FP64 diagnostics of the current state.  Synchronises the stream. */
int mpcd_diagnostics(mpcd_ctx *ctx, mpcd_diag *out, void *stream);

int mpcd_sizes(const mpcd_ctx *ctx, mpcd_sizes_t *out);

/* Message of the sticky error (or "ok").  The string lives in the context. */
const char *mpcd_last_error(const mpcd_ctx *ctx);

/* Capture buffers for tests.  After mpcd_set_debug(ctx, 1) every collision
 * keeps a copy of its cell sums before they are consumed.
 * sums:      [sum_words][n_cells].  P32: int64 words, exact sums over the cell
 *              of per-particle integers: w0 = p_x + 2^48 [solvent],
 *              w1 = p_y + 2^48 [site], w2 = p_z with p = round(fl32(m v) 2^32)
 *              (the low 48 bits of w0 and w1 are the signed momentum sums, the
 *              high 16 bits the cell's solvent and site counts); SRD:
 *              w3 = round(e 2^28), e = fl32(fl32(px vx) + fl32(py vy)) + fl32(pz vz)
 *              in float32; AT: w3, w4, w5 = round(fl32(m xi) 2^32).  The 2^-32
 *              quantum is below the float32 spacing of every |m v| >= 2^-9, so
 *              the momentum words are the exact sums of the stored float32
 *              momenta.  P64: doubles N, M, m v (3), then m v.v (SRD) or m xi
 *              (3) (AT).  The P32 form needs one site mass per context, at most
 *              65535 solvent particles and 65535 sites per cell,
 *              |sum m v_a| < 2^15 per cell, and |m v_a| < 2^14 and
 *              m |v|^2 < 2^27 per particle (the last three not checked).
 * params:    [n_cells][param_bytes] collision parameters (u, kappa, axis / xibar).
 * site_cell: [n_sites] replica-local cell of every site.
 * site_v:    [n_sites][3] site velocities entering the collision (float/double).
 * shift:     [n_replicas][3] integer grid shift S (s = S 2^-20).
 * Any pointer may be NULL.  Synchronises the stream. */
int mpcd_set_debug(mpcd_ctx *ctx, int32_t on);
int mpcd_debug_cells(mpcd_ctx *ctx, void *sums, void *params, int32_t *site_cell, void *site_v,
                     int32_t *shift, void *stream);

/* Per-kernel timing with CUDA events on the launching stream.  While on,
 * mpcd_step() launches kernels one by one (no graph).  get_profile fills up to
 * `max` entries (name, launches, total ms) and returns how many kernels were
 * timed; it synchronises. */
typedef struct {
    char name[48];
    int64_t launches;
    double total_ms;
    double bytes_per_launch;  /* algorithmic bytes moved by one launch */
} mpcd_kernel_time;
int mpcd_set_profiling(mpcd_ctx *ctx, int32_t on);
int mpcd_get_profile(mpcd_ctx *ctx, mpcd_kernel_time *out, int32_t max);
int mpcd_reset_profile(mpcd_ctx *ctx);

/* Per-body velocity autocorrelations (Sec. III.A): C_T(k) = sum over time
 * origins t of V(t).V(t + k) and C_R(k) the same for the space-frame angular
 * velocity omega = Q Ihat^-1 Q^T L, for lags of k = 0 .. n_lags-1 samples, with
 * one sample after every `every`-th step (every sample is a time origin).
 * mpcd_set_vacf(ctx, n_lags, every) clears the sums and starts sampling from the
 * current step; n_lags = 0 stops it.  It synchronises the device.  FP64 on the
 * device, one thread per body, after the POST coupling of each sampled step.
 * mpcd_get_vacf copies the sums, [n_bodies][n_lags] each, and the number of
 * origins summed per lag, [n_lags] (divide to get the averages); any pointer
 * may be NULL; it synchronises the stream and returns MPCD_ERR_ARG while
 * sampling is off. */
#define MPCD_VACF_MAX_LAGS 100000
int mpcd_set_vacf(mpcd_ctx *ctx, int32_t n_lags, int32_t every);
int mpcd_get_vacf(mpcd_ctx *ctx, double *ct, double *cr, int64_t *counts, void *stream);

/* Displacement of every body since the last mpcd_set_state, not wrapped into
 * the box: the sum of the drifts dt P/M of its velocity-Verlet steps (FP64).
 * The long-time self-diffusion coefficient of Sec. III.B (Eq. 15) follows from
 * its mean squared change.  D is a host array of [n_bodies][3] doubles.
 * Synchronises the stream. */
int mpcd_body_displacements(mpcd_ctx *ctx, double *D, void *stream);

/* Constant force f on every body, the sedimentation protocol of Sec. III.B:
 * it acts at the body's centre of mass (the centre site of the paper's spheres;
 * no torque) and a balancing force -B f / N_s acts on every solvent particle,
 * so that the box is force free.  The solvent then streams as
 * v += a dt/2, x += v dt, v += a dt/2 with a = -B f / (N_s m) (exact for a
 * constant force; in the P32 form a dt/2 is rounded to float once and every
 * operation is a float operation in that order); the bodies' velocity-Verlet
 * step includes f.  f = (0, 0, 0) turns it off.  Only contexts with one
 * replica and at least one solvent particle (else MPCD_ERR_ARG).  The bodies'
 * stored forces are recomputed on `stream`. */
int mpcd_set_body_force(mpcd_ctx *ctx, const double f[3], void *stream);

/* Reverse non-equilibrium momentum exchange (Mueller-Plathe), the shear-
 * viscosity protocol of Sec. III.B (Eq. 14).  While enabled, before the
 * collision of every step n with n % period == 0 (after the solvent has
 * streamed to the positions of that collision), the solvent particles of slab A
 * (y in [y_a, y_a + width)) are ranked by |v_x - v_target| and those of slab B
 * (y in [y_b, y_b + width)) by |v_x + v_target|, ascending, ties by particle id;
 * the first min(max_pairs, n_A, n_B) of each list are paired in rank order and
 * exchange v_x.  Slab membership and ranks are decided on the stored values in
 * the context's precision (float for P32: y >= (float)y_a && y < (float)(y_a +
 * width), key fabsf(v_x -+ (float)v_target)).  Each pair moves m (v_A - v_B) of
 * x momentum from slab A to slab B; the totals accumulate on the device.
 * Only contexts with one replica (else MPCD_ERR_ARG).  At most
 * MPCD_RNEMD_MAX_PAIRS pairs.  The candidates of a slab are the particles whose
 * rank key lies at or below the 1/8-octave bucket that holds the max_pairs-th
 * smallest key (keys below 2^-40 share the lowest bucket); if a slab holds more than MPCD_RNEMD_MAX_SLAB particles or more
 * than MPCD_RNEMD_MAX_CANDIDATES candidates, that exchange is skipped and the
 * next synchronising call (e.g. mpcd_rnemd_totals) returns MPCD_ERR_STATE.  enabled = 0 turns the exchange off.  Setting a
 * configuration clears the totals and synchronises the device.  The exchange
 * conserves momentum and kinetic energy exactly.  In mpcd_step the exchange
 * runs after the solvent pass that streamed and binned for the collision, and
 * the exchanged particles' cell words are corrected exactly; mpcd_collide runs
 * it before binning. */
#define MPCD_RNEMD_MAX_PAIRS 1024
#define MPCD_RNEMD_MAX_CANDIDATES 4096
#define MPCD_RNEMD_MAX_SLAB 1048576
typedef struct {
    int32_t enabled;
    int32_t max_pairs;     /* 0 .. MPCD_RNEMD_MAX_PAIRS */
    int32_t period;        /* >= 1 steps */
    int32_t reserved;      /* must be 0 */
    double y_a, y_b;       /* lower edges of slabs A and B, in [0, L_y) */
    double width;          /* slab width (> 0; the slabs must not overlap) */
    double v_target;       /* >= 0 */
} mpcd_rnemd;
int mpcd_set_rnemd(mpcd_ctx *ctx, const mpcd_rnemd *cfg);

/* Totals since the last mpcd_set_rnemd: x momentum moved from slab A to slab B
 * (sum of m (v_A - v_B), FP64) and the number of exchanged pairs.  Synchronises
 * the stream. */
int mpcd_rnemd_totals(mpcd_ctx *ctx, double *p_exchanged, int64_t *n_pairs, void *stream);

/* Velocity profile (Sec. III.B): the solvent of replica 0 binned by the
 * coordinate `bin_axis` into n_bins equal bins over [0, L), and each bin's mass
 * and momentum along `vel_axis` summed in FP64; the bodies add M and P at their
 * centre of mass.  mass and momentum are host arrays of n_bins doubles.
 * Synchronises the stream. */
#define MPCD_PROFILE_MAX_BINS 2048
int mpcd_velocity_profile(mpcd_ctx *ctx, int32_t bin_axis, int32_t vel_axis, int32_t n_bins, double *mass,
                          double *momentum, void *stream);

/* Launch configuration of the solvent pass and the re-sort period.  The
 * autotuner times candidate configurations on the current state (which it
 * restores afterwards) and keeps the fastest: each candidate runs
 * mpcd_step(steps_per_trial) twice from that state, the first run recording its
 * CUDA graph, the second, timed, replaying it; the trials leave the exchange
 * totals and the autocorrelation sums as they were.  set_tuning fixes one directly.
 * Any field <= 0 keeps its current value. */
typedef struct {
    int32_t block;          /* threads per CTA of the solvent pass */
    int32_t tile;           /* particles per work tile */
    int32_t ctas_per_sm;    /* persistent CTAs per SM (capped by shared memory) */
    int32_t sort_period;    /* steps between re-sorts */
    int32_t staged;         /* 1: stage tiles in shared memory with bulk async copies (three-
                               stage ring, one CTA barrier per tile); 2: warp-specialised - a producer warp drives
                               a three-stage ring of bulk copies for the computing warps;
                               3: a three-stage ring per warp (tile = particles per warp tile);
                               0: direct 128-bit loads; -1 keeps the current value */
} mpcd_tuning;
int mpcd_get_tuning(const mpcd_ctx *ctx, mpcd_tuning *out);
int mpcd_set_tuning(mpcd_ctx *ctx, const mpcd_tuning *t);
int mpcd_autotune(mpcd_ctx *ctx, int32_t steps_per_trial, void *stream);

/* ------------------------------------------------------------------------
 * Solvent collision without any device allocation.
 *
 * The paper has no counterpart to this call: it is a library service for
 * callers that must not allocate device memory at the point where they need a
 * collision, e.g. a host code whose framework owns the whole device pool (a
 * new cudaMalloc would fail or fragment it) or a time-critical loop where
 * cudaMalloc/cudaFree would stall (cudaFree synchronises the device).  Such a
 * caller cannot use mpcd_create, which allocates the context's state.
 *
 * One collision (Sec. II.A) of a single periodic box of solvent only, at
 * `step`: random grid shift, binning, exact fixed-point cell sums, then SRD
 * rotation by alpha about a random per-cell axis (with the cell-level
 * thermostat if params->thermostat) or MPCD-AT.  It computes what
 * mpcd_collide computes for a context holding the same box with no colloids
 * at the same step (P32 form; same Philox streams, keyed by params->seed,
 * replica 0, and the particle ids in `tag`).  Positions are not changed;
 * velocities are updated in place.
 *
 * Arguments (device pointers, caller-owned, on the current CUDA device):
 *   params     host struct; precision must be MPCD_P32 and angular 0
 *              (sort_period and naive_transfer are ignored)
 *   L          host int32[3], cells per edge, each 3 to 2047 (the binning
 *              rule forms floor(x 2^20) in 32 bits)
 *   n_solvent  particles, 0 <= n <= MPCD_STATIC_MAX_SOLVENT, a multiple of 4
 *   x, y, z    float[n] positions in [0, L) (not checked)
 *   vx, vy, vz float[n] velocities, updated in place
 *   tag        uint32[n] particle ids (the counter of the MPCD-AT draws);
 *              may be NULL for MPCD_SRD
 *   step       collision index (>= 0), keys the grid shift and all draws
 *   stream     cudaStream_t as void*; the work is enqueued asynchronously
 *   msg        optional host buffer of msg_len bytes for an error message
 * Every device array must be 16-byte aligned.  The P32 per-cell limits of
 * mpcd_debug_cells apply (at most 65535 particles and |sum m v_a| < 2^15 per
 * cell, |m v_a| < 2^14 and m |v|^2 < 2^27 per particle); this call does not
 * check them: a cell beyond them gets wrong
 * velocities and no error is reported.
 *
 * Scratch: the cell sums and collision parameters live in one statically
 * reserved device array of the library (about 5.2 MB per device, reserved by
 * the CUDA runtime when it loads that part of the library on the device, at
 * the latest on the first call), sized for MPCD_STATIC_MAX_CELLS cells.  A box with more cells, more particles than
 * MPCD_STATIC_MAX_SOLVENT, a misaligned pointer or an n that is not a multiple
 * of 4 is rejected with MPCD_ERR_ARG and a message before any device work.  The
 * call allocates nothing; it zeroes the cell sums it uses before binning.  The
 * first call on each device looks up the scratch address (cudaGetSymbolAddress)
 * and the SM count; make that first call before any stream capture begins.
 *
 * The scratch is shared by all calls on a device: calls that overlap in time
 * (other streams, other host threads) race on it and give wrong results.
 * Serialise them, e.g. on one stream.  Returns MPCD_OK, MPCD_ERR_ARG or
 * MPCD_ERR_CUDA (a launch failed). */
#define MPCD_STATIC_MAX_CELLS 65536
#define MPCD_STATIC_MAX_SOLVENT 4194304
int mpcd_collide_solvent_static(const mpcd_params *params, const int32_t L[3], int64_t n_solvent,
                                const float *x, const float *y, const float *z, float *vx,
                                float *vy, float *vz, const uint32_t *tag, int64_t step,
                                void *stream, char *msg, size_t msg_len);

#ifdef __cplusplus
}
#endif
#endif /* MPCD_H */
