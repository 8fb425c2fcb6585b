/*
 * mdf.h -- C-ABI of the GB300 (sm_103a) MDF-LBM library.
 *
 * The library advances the multiple-distribution-function lattice Boltzmann
 * method of Chai, Shi & Zhan (arXiv 2108.08591) for the incompressible
 * Navier-Stokes equations written as d+1 coupled convection-diffusion
 * equations (Eq. 2-2): one D2Q5 (2D) or D3Q7 (3D) distribution set per
 * equation, the MRT collision Lambda = M^-1 S_d M (Eq. 4-1 .. 4-3) and the
 * evolution of Eq. 3-21 (diffusive scaling, lattice units dx = dt = c = 1).
 * Options: the D2Q4 / D3Q6 lattices (Sec. 2.2), Scheme II forcing (Eq. 2-3c),
 * a non-equilibrium start (the inverse of Eq. 3-16), the in-place AA stream
 * (one population buffer) and a slab decomposition with its face exchange.
 *
 * Conventions shared by every entry point:
 *   - Every call returns an mdf_status; nothing aborts the process.  On an
 *     error, mdf_last_error(h) (or mdf_last_error(NULL) for a failed create)
 *     returns a human-readable message.
 *   - Node order is x fastest: n = x + nx*(y + ny*z).  A scalar field is
 *     [N] doubles, a vector field [d][N], with N = nx*ny*nz and no padding.
 *   - Device pointers passed in are owned by the caller and must stay valid
 *     until the work enqueued on the library's stream has finished.
 *   - All GPU work is enqueued on the stream given at create time (stream
 *     ordered, asynchronous) unless a function says it synchronises.
 *   - Lattice units: x_j = j, dt = 1; P0 = rho0 = 1 is the rest state.
 */
#ifndef MDF_H
#define MDF_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mdf_s *mdf_t;

typedef enum {
    MDF_OK = 0,
    MDF_EINVAL = 1,          /* bad argument (null, size, rate outside (0,2), ...) */
    MDF_ENOMEM = 2,          /* device or host allocation failed */
    MDF_ECUDA = 3,           /* a CUDA call failed; see mdf_last_error */
    MDF_EDIVERGED = 4,       /* a reduction met a non-finite value */
    MDF_ETIMEOUT = 5,        /* a bounded device wait gave up */
    MDF_ENOTCONVERGED = 6,   /* step cap reached before the tolerance */
    MDF_EUNSUPPORTED = 7,    /* valid but not built (lattice, storage, ...) */
    MDF_EIO = 8              /* checkpoint file error or checksum mismatch */
} mdf_status;

/* Population storage.  All collision arithmetic is FP32 except for MDF_F64
 * (FP64 throughout).
 *   MDF_F32, MDF_F16, MDF_BF16, MDF_F64: populations stored shifted by the
 *     rest state f_rest = f^eq(P0 = 1, u = 0) (Eq. 2-4), so the stored
 *     numbers are O(U) instead of O(1).
 *   MDF_F16EQ, MDF_BF16EQ: equilibrium-shifted 16-bit storage: each node keeps
 *     its post-collision non-equilibrium part f* - f^eq(M) in 16 bits (FP16
 *     scaled by 2^14) plus its moments M = (u, P - P0[, rho - rho0]) in FP32;
 *     a pull adds back f^eq of the source node's M.  The 16-bit rounding then
 *     falls on f^ne only, so P and the Eq. 3-16 gradients stay accurate.
 *     Bytes per node update: 4 q nsets + 8 (d + 1 + with_rho). */
enum { MDF_F32 = 0, MDF_F16 = 1, MDF_BF16 = 2, MDF_F64 = 3, MDF_F16EQ = 4, MDF_BF16EQ = 5 };

/* Where a caller's array lives. */
enum { MDF_HOST = 0, MDF_DEVICE = 1 };

typedef struct {
    int nx, ny, nz;          /* nodes per axis; nz = 1 when d = 2 */
} mdf_grid;

typedef struct {
    double s0, s1, s2;       /* S_d = diag(s0, s1.., s2..) of Eq. 4-3; s2 < 0 selects
                                the paper's rule s2 = 8(2 - s1)/(8 - s1) (Sec. 4.1).
                                Viscosity nu = (1/s1 - 1/2) c_s^2 (Eq. 3-13a). */
} mdf_rates;

typedef struct {
    int wall[3];             /* per axis: 0 periodic, 1 halfway walls at both ends */
    int lid;                 /* 1: the + face of the last axis moves with lid_u */
    double lid_u[3];         /* lid velocity (lattice units) */
} mdf_bc;

typedef struct {
    int storage;             /* one of the MDF_F32 .. MDF_BF16EQ storage types */
    int with_rho;            /* 1: also carry the alpha = 0 (continuity) set, so d+1
                                sets are advanced; 0: only the d velocity sets (the
                                paper shows alpha = 0 can be omitted, Sec. 3.2) */
    void *stream;            /* cudaStream_t to enqueue on; NULL = legacy default */
    int vx;                  /* x-nodes per thread of the update kernel: 0 = tuned
                                default; 1 = one node per thread; 2, 4, 8 = vector
                                widths (FP32: 2, 4; FP16/BF16: 4, 8; FP64: 2;
                                *EQ: 2, 4).  In 3D, where wider kernels spill
                                registers, requests are clamped to 4 (rest-shifted
                                16-bit, FP64) or 2 (FP32, *EQ);
                                mdf_info reports the width in use.  A width that
                                does not divide nx falls back to 1. */
    int block;               /* threads per block of the update kernel: 0 = tuned
                                default, else a multiple of 32 in [32, 256] */
    int q;                   /* directions per set: 0 = D2Q5 / D3Q7 (default), 4 = D2Q4,
                                6 = D3Q6 (Sec. 2.2: no rest direction, fewer bytes
                                per node; the rest-shifted storage types only) */
    int inplace;             /* 1: one population buffer, streamed in place by the AA
                                pattern (even updates collide within a node, odd
                                updates read and write the neighbours; same results
                                as the default pull stream over two buffers, half
                                the population memory).  Rest-shifted storage types
                                only; one node per thread; no mdf_autotune. */
} mdf_opts;

/* Derived-field outputs, each a caller-owned array of doubles or NULL.
 * Layout (N nodes, d dimensions):
 *   P[N]        pressure, Eq. 3-15 (R = 0)
 *   u[d][N]     velocity, Eq. 2-7
 *   rho[N]      zeroth moment of the alpha = 0 set (needs with_rho = 1)
 *   G[d][d][N]  G[a][b] = du_a/dx_b, Eq. 3-16
 *   div[N]      velocity divergence, Eq. 3-16a
 *   S[k][N]     strain rate, Eq. 3-17, upper triangle in row order
 *               (2D: xx, xy, yy; 3D: xx, xy, xz, yy, yz, zz)
 *   sigma[k][N] shear stress, Eq. 3-17a, same order (rho0 = 1)
 *   omega[.][N] vorticity, Eq. 3-18/3-19: 2D du2/dx - du1/dy; 3D (wx, wy, wz)
 * where = MDF_DEVICE: device pointers, filled asynchronously.
 * where = MDF_HOST: host pointers; the call stages through device memory
 * and synchronises the stream before returning. */
typedef struct {
    double *P, *u, *rho, *G, *div, *S, *sigma, *omega;
    int where;
} mdf_fields_t;

/* Static facts about a handle. */
typedef struct {
    int d, q, nsets, storage;
    int nx, ny, nz, pitch;   /* pitch: padded x extent of the device arrays */
    long long nodes;         /* nx*ny*nz */
    long long step;          /* time steps taken since the last init/load */
    double bytes_per_update; /* algorithmic bytes per node update: one read and one
                                write of every population (2 q nsets sizeof(T)) */
    double s0, s1, s2;
    int vx, block;           /* launch shape of the update kernel in use */
} mdf_info_t;

/*
 * mdf_create -- allocate a lattice of d+1 (or d) distribution sets.
 *   g: grid (nx, ny >= 2; nz = 1 for d = 2, nz >= 2 for d = 3);
 *   d: 2 (D2Q5, Sec. 2.2) or 3 (D3Q7, Sec. 2.2, MRT basis read analogously
 *      to Eq. 4-2); o->q = 4 or 6 selects D2Q4 or D3Q6 (Sec. 2.2), with the
 *      conserved, first-moment and traceless second-moment rows as basis;
 *   r: relaxation rates, each in (0, 2);
 *   bc: periodic axes or anti-halfway bounce-back walls (Sec. 4), optional
 *      moving lid;  o: storage, sets and stream.
 * The library allocates and owns the population buffers (two of
 * 2*q*nsets*pitch*ny*nz elements), the link mask and its scratch.  The state
 * is undefined until mdf_init or mdf_load.  Errors: MDF_EINVAL,
 * MDF_EUNSUPPORTED, MDF_ENOMEM, MDF_ECUDA; *h is NULL on error.
 */
mdf_status mdf_create(mdf_t *h, const mdf_grid *g, int d, const mdf_rates *r,
                      const mdf_bc *bc, const mdf_opts *o);

/* Release every resource of h (synchronises its stream).  NULL is ignored. */
void mdf_destroy(mdf_t h);

/*
 * mdf_init -- set f = f^eq(P, u) at every node (Sec. 4: initialisation by
 * the equilibrium of Eq. 2-4), for the alpha = 0 set with ubar_0 = rho0 = 1.
 *   P[N], u[d][N]: FP64 arrays in `where` memory (MDF_HOST or MDF_DEVICE).
 * Resets the step counter.  Host arrays are copied before the call returns;
 * device arrays must stay valid until the stream reaches this work.
 */
mdf_status mdf_init(mdf_t h, const double *P, const double *u, int where);

/*
 * mdf_init_neq -- as mdf_init, plus the first-order non-equilibrium part of
 * a given velocity gradient, so that the start has no initial layer:
 *   f^ne_{i,alpha} = -(dt / s1) w_i c_i . (G_alpha - (tr G / d) e_alpha)
 * for alpha = 1..d, and none for alpha = 0.  This is the inverse of
 * Eq. 3-16: the fields of the new state give back the traceless part of G.
 * The trace is dropped because Eq. 3-15 would read it as pressure, so P is
 * kept.
 *   G[a][b][N] = du_a / dx_b (lattice units): FP64 in `where` memory, laid
 *     out like mdf_fields_t.G.  Same ownership rules as P and u.
 * Errors: MDF_EINVAL for a null G, plus those of mdf_init.
 */
mdf_status mdf_init_neq(mdf_t h, const double *P, const double *u, const double *G, int where);

/*
 * mdf_set_force -- body force Fbar_alpha(x) of Eq. 2-6 (F_i = w_i Fbar_alpha),
 * added as dt w_i Fbar_alpha in Eq. 3-21.  F[d][N] FP64 in `where` memory,
 * stored on the device in the compute precision (FP32; FP64 for MDF_F64
 * storage); NULL removes the force.
 */
mdf_status mdf_set_force(mdf_t h, const double *F, int where);

/*
 * mdf_set_forcing -- forcing scheme of the update (Sec. 3.2):
 *   MDF_FORCING_EQ321   (default) Eq. 3-21: f* = f - Lambda (f - f^eq) + dt F;
 *   MDF_FORCING_SCHEME2 Scheme II, Eq. 2-3c and Eq. 2-7a: the state is
 *     fbar = f - dt F/2, fbar* = fbar - Lambda (fbar - f^eq) + dt (I - Lambda/2) F,
 *     ubar_alpha = sum_i fbar_{i,alpha} + dt Fbar_alpha / 2, and P from
 *     Eq. 3-15 over fbar.
 * Under Scheme II:
 *   - the anti-halfway bounce-back acts on fbar;
 *   - mdf_init stores fbar = f^eq(P, u) - dt F/2 with the force set at
 *     that time, so call mdf_set_force first;
 *   - the fields, sums and residual read ubar from Eq. 2-7a;
 *   - the f^ne of Eq. 3-16 is that of f = fbar + dt F/2, which has the same
 *     first moment.
 * Without a force the two schemes are the same update.  A change does not
 * convert the state; checkpoints record the scheme, and mdf_load requires a
 * match.  Errors: MDF_EINVAL for an unknown scheme.
 */
#define MDF_FORCING_EQ321 0
#define MDF_FORCING_SCHEME2 2
mdf_status mdf_set_forcing(mdf_t h, int scheme);
mdf_status mdf_get_forcing(mdf_t h, int *scheme);

/* mdf_step -- advance n >= 0 time steps of Eq. 3-21 with streaming. */
mdf_status mdf_step(mdf_t h, long long n);

/*
 * mdf_step_fields -- advance n >= 1 steps; the first update also writes the
 * derived fields (Eq. 2-7, 3-15 .. 3-19) of the state it starts from, in the
 * same pass over memory.  Equivalent to mdf_fields(h, out) followed by
 * mdf_step(h, n).  out->where must be MDF_DEVICE.
 */
mdf_status mdf_step_fields(mdf_t h, long long n, const mdf_fields_t *out);

/* mdf_fields -- derived fields of the current state (no step taken). */
mdf_status mdf_fields(mdf_t h, const mdf_fields_t *out);

/*
 * mdf_fields_host_noalloc -- like mdf_fields() with out->where = MDF_HOST,
 * but it allocates nothing.  (This is a library service; the paper has no
 * counterpart.)  mdf_fields() stages host readbacks through a device buffer
 * that the handle grows with cudaMalloc when needed.  Callers that cannot
 * let the library allocate at that moment use this entry point instead:
 * processes whose GPU memory is fully reserved by another allocator (a
 * framework's caching pool, an MPS memory quota), or code that runs while
 * allocation is forbidden, e.g. while another thread captures a CUDA graph
 * in global capture mode.  The fields are staged in one fixed 16 MiB device
 * buffer compiled into the library (2,097,152 doubles), which every GPU that
 * loads the library holds until the process exits.
 *   out: host arrays, out->where must be MDF_HOST; layout as mdf_fields_t.
 * Limits and behaviour:
 *   - the requested fields together may hold at most 2,097,152 doubles
 *     (e.g. P and u of a 2D lattice up to 699,050 nodes); larger requests
 *     return MDF_EINVAL with a message and do nothing;
 *   - the first call on a GPU looks up that buffer's device address (a
 *     one-time set-up per GPU); make that first call before any stream
 *     capture begins;
 *   - every call on a GPU shares the one buffer, which keeps the last call's
 *     contents.  Each call writes every requested field in full before
 *     reading it back, so nothing needs clearing, but calls that overlap on
 *     the GPU (from several threads or streams at once) race on the buffer:
 *     serialise them.  The call synchronises h's stream before returning.
 *   - like every entry point, call it with h's GPU current.
 */
mdf_status mdf_fields_host_noalloc(mdf_t h, const mdf_fields_t *out);

/*
 * mdf_moments -- the macroscopic fields of the current state (no step taken):
 *   P[N]     pressure, Eq. 3-15 with R = 0;
 *   u[d][N]  velocity u_alpha = sum_i f_{i,alpha}, Eq. 2-7 (Eq. 2-7a under
 *            Scheme II);
 *   rho[N]   sum_i f_{i,0} of the alpha = 0 set, a diagnostic (nullable;
 *            ignored when the set is not carried).
 * Caller-owned DEVICE arrays of FP64, x-fastest, laid out as mdf_fields_t.
 * The outputs are FP64 (not FP32) so that P, which sits near P0 = 1, keeps
 * the digits of its O(U^2) fluctuation; the arithmetic is that of the
 * storage type.  Stream-ordered on h's stream.  Same as mdf_fields with only
 * these pointers set.  Errors: MDF_EINVAL for a null P or u.
 */
mdf_status mdf_moments(mdf_t h, double *P, double *u, double *rho);

/*
 * mdf_gradients -- the derived fields of Eq. 3-16 .. 3-19 from the first
 * moment of f^ne = f - f^eq of the current state (no step taken):
 *   G[d][d][N]  du_a/dx_b (Eq. 3-16), div[N] (Eq. 3-16a),
 *   S[k][N]     strain rate (Eq. 3-17), sigma[k][N] viscous stress with
 *               rho0 = 1 (Eq. 3-17a), k over the d(d+1)/2 pairs a <= b,
 *   omega[.][N] vorticity (Eq. 3-18, 3-19): one component in 2D, three in 3D.
 * Caller-owned DEVICE arrays of FP64 (see mdf_moments); each pointer is
 * nullable, and at least one must be set (else MDF_EINVAL).
 * Stream-ordered on h's stream; same as mdf_fields with these pointers set.
 */
mdf_status mdf_gradients(mdf_t h, double *G, double *div, double *S, double *sigma,
                         double *omega);

/*
 * mdf_sums -- sums[a] = sum over nodes of ubar_alpha (Eq. 2-7) for every
 * carried set a (alpha = 0 first when with_rho = 1), reduced in FP64 in a
 * fixed order (deterministic).  sums: host array of nsets doubles.
 * Synchronises the stream.  MDF_EDIVERGED if a value is not finite.
 */
mdf_status mdf_sums(mdf_t h, double *sums);

/*
 * mdf_residual -- steady-state residual r = ||u - u_prev||_2 / ||u||_2 over
 * all nodes in FP64, where u_prev is the velocity at the previous
 * mdf_residual call (r = +inf on the first call after init/load).  *r on the
 * host.  Synchronises.  MDF_EDIVERGED if u is not finite.
 */
mdf_status mdf_residual(mdf_t h, double *r);

/* mdf_mask -- link mask [N] bytes to host memory: bit i set when the link
 * from the node along c_i crosses a wall; bit 7 when it crosses the lid.
 * Synchronises. */
mdf_status mdf_mask(mdf_t h, unsigned char *host_out);

/* mdf_save / mdf_load -- raw populations plus a header (grid, d, q, sets,
 * storage, rates, boundary, forcing scheme, buffer layout and AA parity,
 * step) and an FNV-1a checksum.  Load requires a handle created with the
 * same configuration; MDF_EIO on a mismatch or a corrupt file.  Both
 * synchronise.  A resumed run is bit-identical. */
mdf_status mdf_save(mdf_t h, const char *path);
mdf_status mdf_load(mdf_t h, const char *path);

/* mdf_info -- static facts about h (host struct). */
mdf_status mdf_info(mdf_t h, mdf_info_t *out);

/*
 * mdf_autotune -- measure the update kernel's launch shapes for this handle
 * (one node per thread and each vector width built for the storage type
 * that divides nx, times 64/128/256 threads per block; `reps` timed updates
 * each, CUDA events on h's stream) and keep the fastest.  The candidates
 * update out of place without advancing the state, so the lattice is left
 * as it was.  *vx, *block (nullable) receive the choice.  Synchronises.
 */
mdf_status mdf_autotune(mdf_t h, int reps, int *vx, int *block);

/*
 * Slab decomposition (one lattice as k sub-domains on one GPU).
 *
 * mdf_slabs_create -- split the grid g along its last axis (y in 2D, z in 3D)
 * into k equal slabs, each a lattice of its own with one ghost layer on
 * either side.  After every update, mdf_slabs_step copies device to device,
 * per face and set, the one layer of post-collision populations that points
 * across the face (the direction along +axis into the upper neighbour's
 * lower ghost layer and the one along -axis into the lower neighbour's
 * upper ghost layer).  This is the exchange that ranks holding neighbouring
 * slabs would make.  The results equal the undivided lattice's bit for bit.
 *   - The split axis must be periodic.  The two-buffer rest-shifted storage
 *     types only.  All slabs use o->stream.
 *   - Errors: MDF_EINVAL (k does not divide the axis), MDF_EUNSUPPORTED, and
 *     those of mdf_create.
 * mdf_slabs_init   -- f = f^eq(P, u) from global host arrays (as mdf_init).
 * mdf_slabs_step   -- n updates with the exchange after each.
 * mdf_slabs_fields -- the derived fields of the global lattice, host outputs
 *                     only (out->where = MDF_HOST); synchronises.
 */
typedef struct mdf_slabs_s *mdf_slabs_t;
mdf_status mdf_slabs_create(mdf_slabs_t *s, const mdf_grid *g, int d, const mdf_rates *r,
                            const mdf_bc *bc, const mdf_opts *o, int k);
mdf_status mdf_slabs_init(mdf_slabs_t s, const double *P, const double *u);
mdf_status mdf_slabs_step(mdf_slabs_t s, long long n);
mdf_status mdf_slabs_fields(mdf_slabs_t s, const mdf_fields_t *out);
void mdf_slabs_destroy(mdf_slabs_t s);
const char *mdf_slabs_last_error(mdf_slabs_t s);

/* mdf_sync -- wait for all work enqueued on h's stream. */
mdf_status mdf_sync(mdf_t h);

/* mdf_last_error -- message of the last failure on h (NULL: of the calling
 * thread's last failed mdf_create).  Never NULL. */
const char *mdf_last_error(mdf_t h);

/* ------------------------------------------------------------------------
 * Batched lid-driven cavities (the cavity of Sec. 4.3 in lattice units).
 *
 * Many closed boxes of different sides and Reynolds numbers advanced
 * together to steady state: anti-halfway bounce-back on every wall, the +
 * face of the last axis (the lid) moving along x with `lid_speed`;
 * nu = lid_speed * side / Re, s1 from Eq. 3-13a, s2 from the rule of
 * Sec. 4.1; FP32 rest-shifted storage (opts->storage must be MDF_F32).  All
 * nodes share one pool, tiled 128 nodes per tile, and one persistent
 * cooperative kernel per convergence period walks the tiles of the cavities
 * still running with a bounded grid barrier between steps (a barrier that
 * waits more than ~2 s returns MDF_ETIMEOUT instead of hanging).
 * ------------------------------------------------------------------------ */
typedef struct mdf_batch_s *mdf_batch_t;

/* mdf_batch_create -- n cavities (1 .. 8192) of dimension d (2: D2Q5 squares,
 * 3: D3Q7 cubes), side[c] fluid nodes per axis, Reynolds number Re[c].
 * The state is the rest state after mdf_batch_init(b, -1, NULL, NULL, 0). */
mdf_status mdf_batch_create(mdf_batch_t *b, int d, int n, const int *side, const double *Re,
                            double lid_speed, const mdf_opts *o);
void mdf_batch_destroy(mdf_batch_t b);

/* mdf_batch_init -- cavity c (or all when c = -1) to f = f^eq(P, u): P[N^d],
 * u[d][N^d] FP64 in `where` memory, or the rest state when P = u = NULL. */
mdf_status mdf_batch_init(mdf_batch_t b, int cavity, const double *P, const double *u, int where);

/* mdf_batch_seed -- as mdf_batch_init; with neq = 1 (P and u required) the
 * velocity sets also get the first-order non-equilibrium part of the seed,
 * f^ne_i = -(w_i / s1) [(c_i . grad) u_alpha - c_{i,alpha} div u / d] (the
 * Chapman-Enskog term whose first moment Eq. 3-16 maps back to grad u, made
 * traceless so that Eq. 3-15 still returns P), with grad u by central
 * differences of u and ghost values 2 u_wall - u beyond the walls.  The
 * initial state then has the seed's u and P, and its Eq. 3-16 gradient is
 * the traceless part of that finite-difference gradient. */
mdf_status mdf_batch_seed(mdf_batch_t b, int cavity, const double *P, const double *u, int where, int neq);

/* mdf_batch_run -- advance every cavity until its residual
 * r = ||u^n - u^{n-R}||_2 / (R ||u^n||_2), the mean per-step relative change
 * of u over the check period R = check_every (even), computed in FP64, drops
 * below tol, it diverges, or it has taken max_steps steps.  Per cavity (host arrays of n, each nullable): steps
 * taken, status (MDF_OK converged, MDF_EDIVERGED, MDF_ENOTCONVERGED) and
 * the last residual.  Returns MDF_OK when every cavity converged, else the
 * first non-OK status.  Synchronises; a period is one captured CUDA graph
 * when the stream is not the legacy default stream. */
mdf_status mdf_batch_run(mdf_batch_t b, double tol, long long max_steps, int check_every,
                         long long *steps, int *status, double *res);

/* mdf_batch_step -- advance every cavity by n steps (no convergence checks). */
mdf_status mdf_batch_step(mdf_batch_t b, long long n);

/* mdf_batch_fields -- derived fields (Eq. 2-7, 3-15 .. 3-19) of one cavity,
 * layout as mdf_fields_t with N = side^d nodes. */
mdf_status mdf_batch_fields(mdf_batch_t b, int cavity, const mdf_fields_t *out);

/* mdf_batch_info -- total fluid nodes, tiles and persistent-grid blocks. */
mdf_status mdf_batch_info(mdf_batch_t b, long long *nodes, int *tiles, int *grid);

/* mdf_batch_set_timeout -- spin limit of the grid barrier in SM clock cycles
 * (default 4e9, about 2 s).  A barrier that waits longer makes every block of
 * the persistent kernel return and the call report MDF_ETIMEOUT; the batch
 * state is then undefined until the next mdf_batch_init. */
mdf_status mdf_batch_set_timeout(mdf_batch_t b, long long cycles);

/* Scheduling of the batch's persistent kernel (mdf_batch_set_schedule,
 * mdf_batch_get_schedule, mdf_batch_autotune) is a GPU launch control with
 * no counterpart in the paper: it changes how the updates of Eq. 3-21 are
 * distributed over the GPU, never their arithmetic.
 *
 * mdf_batch_set_schedule -- launch shape of the persistent step kernel:
 * `threads` per block in {32, 64, 128} (each thread updates 128 / threads
 * nodes of a 128-node tile, `threads` apart), `grid` co-resident blocks (0:
 * the most that fit, MDF_EINVAL above that) and `sched` 0 (live tiles dealt
 * round-robin to the blocks, a grid barrier between steps), 1 (one
 * contiguous run of tiles per block, grid barrier), 2 (round-robin, no
 * grid barrier: a tile starts a step once the tiles within one neighbour
 * stride of it have finished the previous one) or 3 (round-robin but for
 * the last eight rounds of each step, whose tiles the blocks claim one at a
 * time from an atomic ticket counter; grid barrier).  Every schedule
 * computes the same bits; only the speed differs.  MDF_EINVAL for other
 * values.  A new batch starts with 64 threads, schedule 3 and the largest
 * grid. */
mdf_status mdf_batch_set_schedule(mdf_batch_t b, int threads, int grid, int sched);

/* mdf_batch_get_schedule -- the launch shape in use (any pointer may be NULL). */
mdf_status mdf_batch_get_schedule(mdf_batch_t b, int *threads, int *grid, int *sched);

/* mdf_batch_autotune -- time `reps` (rounded up to even; < 2: 20) steps of
 * every schedule candidate (threads 128 / 64 / 32, schedules 0 .. 3, grids
 * of 1, 2, 3, 4, 6, 8, 12, 16, 24, 32 blocks per SM up to the co-resident limit) on
 * the current state with all cavities live, keep the fastest and restore
 * the state (bit for bit; step counts and statuses are not touched).
 * Needs one extra population pool of device memory while it runs. */
mdf_status mdf_batch_autotune(mdf_batch_t b, int reps, int *threads, int *grid, int *sched);

/* mdf_batch_last_error -- message of the last failure (NULL: last create). */
const char *mdf_batch_last_error(mdf_batch_t b);

/* ------------------------------------------------------------------------
 * Learned warm start: a U-Net mapping cavity parameters to an approximate
 * steady (P - P0, u, v) field that seeds mdf_batch_init.  Not part of the
 * paper's method: a data-driven initial state for it.  Trained on the GPU by
 * the library's own BF16 tensor-core convolution kernels (FP32
 * accumulation, FP32 master weights, Adam).
 *   level l = 0 .. levels-1 (channels[l]): two 3x3 convolutions with ReLU,
 *     2x2 average pooling between levels; decoder: nearest 2x upsampling,
 *     concatenation with the encoder output of the level, two convolutions
 *     with ReLU; head: one linear 3x3 convolution to `cout` channels.
 * Tensors are NHWC FP32 on the device: x[B][H][W][cin] (unused input
 * channels zero), y[B][H][W][cout]; targets t[B][H][W][cout_used].
 * ------------------------------------------------------------------------ */
typedef struct mdf_ws_s *mdf_ws_t;

/* H, W divisible by 2^(levels-1); cin, cout, channels[] multiples of 16;
 * weights He-uniform from SplitMix64(seed), biases 0; buffers for up to
 * max_batch samples; work on `stream` (cudaStream_t, may be NULL). */
mdf_status mdf_ws_create(mdf_ws_t *w, int H, int W, int levels, const int *channels, int cin,
                         int cout, int cout_used, int max_batch, unsigned long long seed,
                         void *stream);
void mdf_ws_destroy(mdf_ws_t w);
long long mdf_ws_param_count(mdf_ws_t w);
/* Parameters (FP32) per convolution in forward order e0a, e0b, ..,
 * e{L-1}b, d{L-2}a, d{L-2}b, .., d0a, d0b, head: weights [Cout][3][3][Cin]
 * then biases.  get: parameters and the last gradients to host (nullable). */
mdf_status mdf_ws_get_params(mdf_ws_t w, float *host, float *grad_host);
/* set: parameters from host; resets the Adam moments. */
mdf_status mdf_ws_set_params(mdf_ws_t w, const float *host);
/* y = net(x) for B <= max_batch samples (device pointers). */
mdf_status mdf_ws_forward(mdf_ws_t w, const float *x, int B, float *y);
/* One step: forward, MSE loss against t, backward, and (lr > 0) Adam with
 * beta = (0.9, 0.999), eps = 1e-8.  *loss (nullable, host) gets the loss;
 * asking for it synchronises. */
mdf_status mdf_ws_train_step(mdf_ws_t w, const float *x, const float *t, int B, float lr,
                             double *loss);
const char *mdf_ws_last_error(mdf_ws_t w);

/* The network's convolution kernels on caller-owned device buffers (NHWC
 * BF16 activations, [Cout][3][3][Cin] BF16 weights; Cin, Cout % 8 == 0):
 *   fwd:   y = conv(x) + bias (ReLU if relu), to y (BF16) and/or yf (FP32);
 *   wgrad: dw[Cout][9 Cin] (FP32) = sum over pixels of dz x im2col(x), with
 *          `part` a scratch of mdf_nn_wgrad_scratch(...) floats;
 *   dgrad: dx (BF16) = gradient of the input for dz, with `wt` a BF16 scratch
 *          of Cout * 9 * Cin elements. */
mdf_status mdf_nn_conv_fwd(const void *x, const void *w, const float *bias, void *y, float *yf,
                           int B, int H, int W, int Cin, int Cout, int relu, void *stream);
long long mdf_nn_wgrad_scratch(int B, int H, int W, int Cin, int Cout);
mdf_status mdf_nn_conv_wgrad(const void *x, const void *dz, float *dw, float *part, int B, int H,
                             int W, int Cin, int Cout, void *stream);
mdf_status mdf_nn_conv_dgrad(const void *dz, const void *w, void *wt, void *dx, int B, int H, int W,
                             int Cin, int Cout, void *stream);
/* Forward/dgrad convolution kernel, process-wide: which = 2 the tcgen05
 * kernel with one staged input halo per channel chunk reused by the nine
 * taps (the default; Cin % 16 != 0 falls back to 1), 1 the tcgen05 kernel
 * with im2col gathers, 0 the mma.sync kernel.  All accumulate in FP32. */
mdf_status mdf_nn_set_conv_kernel(int which);

/* Tile of the tcgen05 kernel, process-wide: bn (output channels per CTA) in
 * {16, 32, 64, 128, 256} and stages (shared-memory ring depth) in {3, 4, 6};
 * 0 keeps the automatic choice.  (256, 6) does not fit and is rejected.
 * A tuning override: every tile sweeps K in the same order. */
mdf_status mdf_nn_set_tc_tile(int bn, int stages);

/* Tile of the halo kernel, process-wide: mt 128-output M tiles per CTA (1 or
 * 2) and kc input channels per staged chunk (16 or 32, used when it divides
 * Cin); 0 keeps the automatic choice.  Its N tile follows
 * mdf_nn_set_tc_tile's bn. */
mdf_status mdf_nn_set_halo_tile(int mt, int kc);

/* Weight-gradient kernel, process-wide: which = 1 the tcgen05 kernel (the
 * default: TMA-loaded dz and shifted x boxes, the taps of one kernel row
 * per CTA in three TMEM accumulators, M = output channels, or input
 * channels where that pads fewer of the 128 rows and Cout % 32 == 0;
 * Cin % 16 != 0 or Cout % 8 != 0 falls back to 0), 0 the mma.sync split-K
 * kernel.  Both accumulate in FP32. */
mdf_status mdf_nn_set_wgrad_kernel(int which);

/* Launch shape of the tcgen05 weight-gradient kernel, process-wide: N tile
 * bn 16, 32 or 64 channels (of Cin, or of Cout where the roles are
 * swapped; a tile that does not divide them falls back to the largest that
 * does; 0 keeps the automatic choice, the largest that divides), the
 * CTAs per SM that its pipeline depth leaves shared memory for (1 .. 16; 0
 * keeps the default 3) and the pixel positions per pipeline stage kc, 64
 * or 128 (0: 128); the pixel split fills one wave of the CTAs that fit.
 * MDF_EINVAL otherwise. */
mdf_status mdf_nn_set_wgrad_tile(int bn, int ctas_per_sm, int kc);

/* Read and clear the tcgen05 kernel's time-out flag (1 when a bounded
 * mbarrier wait gave up) of the current device; synchronises the device. */
mdf_status mdf_nn_conv_error(int *flag);

#ifdef __cplusplus
}
#endif
#endif /* MDF_H */
