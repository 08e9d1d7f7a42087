/*
 * klb.h -- C ABI of the GB300 library for the three-species Keldysh-lattice
 * Boltzmann (KLB) step: water ("hydron") populations in a nanochannel,
 * electron and phonon populations in its solid walls (Sec. 4 of Succi &
 * Montessori, "Keldysh-Lattice Boltzmann approach to quantum nanofluidics").
 *
 * Conventions used by every entry point
 * -------------------------------------
 * - Plain C types only.  Device memory is passed as void* (any cudaMalloc'd or
 *   torch-allocated buffer on the current device); host arrays as plain
 *   pointers.  The caller owns every buffer it passes; the library owns only
 *   the handle and small host tables, and never calls cudaMalloc/cudaFree.
 * - Errors are returned as klb_status; nothing is thrown across the ABI.
 *   klb_last_error() gives the message of the last failing call on a handle.
 * - One handle is used by one host thread at a time.  Work is enqueued on the
 *   handle's CUDA stream; only calls documented as synchronising wait for it.
 * - Dense host arrays ("box layout") index cell (x, y, z) as
 *   x + nx * (y + ny * z), x fastest.  Arrays with a leading species index
 *   use the order water (0), electron (1), phonon (2); arrays with a
 *   component index use x, y, z.  Entries of cells that do not carry a
 *   species are written as 0 and ignored on input.
 * - Populations are deviations g_i = f_i - w_i rho0 from the rest state, in
 *   the direction order: D2Q9 as numbered in Sec. 4.2 (0 rest, 1 right,
 *   2 up, 3 left, 4 down, 5 right-up, 6 left-up, 7 left-down, 8 right-down);
 *   D3Q19: 0 rest, (+x,-x,+y,-y,+z,-z), then (1,1,0), (-1,-1,0), (1,-1,0),
 *   (-1,1,0), (1,0,1), (-1,0,-1), (1,0,-1), (-1,0,1), (0,1,1), (0,-1,-1),
 *   (0,1,-1), (0,-1,1).
 */
#ifndef KLB_H
#define KLB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct klb_lattice klb_lattice; /* opaque, library-owned host handle */

typedef enum {
    KLB_OK = 0,
    KLB_EINVAL = 1,    /* bad argument, shape, parameter or buffer size      */
    KLB_ENOMEM = 2,    /* caller buffer too small, or host allocation failed */
    KLB_ECUDA = 3,     /* a CUDA call failed (message in klb_last_error)      */
    KLB_EUNSTABLE = 4, /* a non-finite value was seen                         */
    KLB_ETIMEOUT = 5,  /* reserved for step/time limits of callers            */
    KLB_ESTATE = 6,    /* call not valid in the handle's current state        */
    KLB_ERANGE = 7     /* a 16-bit population difference left its range and
                          was stored saturated (see klb_obs.clipped)          */
} klb_status;

enum { KLB_D2Q9 = 9, KLB_D3Q19 = 19 };
enum { KLB_GEOM_SLAB = 0, KLB_GEOM_PIPE = 1, KLB_GEOM_MASK = 2 };
enum { KLB_FP64 = 0, KLB_FP32 = 1, KLB_FP16_DEV = 2, KLB_BF16_DEV = 3 };
enum { KLB_IFACE_SPECULAR = 0, KLB_IFACE_BOUNCEBACK = 1 };
enum { KLB_WATER = 0, KLB_ELECTRON = 1, KLB_PHONON = 2 };
enum { KLB_PHONON_FLUID = 0, KLB_PHONON_WAVE = 1 };

/*
 * Problem description (Sec. 2 set-up: water driven by a pressure gradient
 * through a nanochannel with solid walls; x is the channel axis and is
 * periodic, Sec. 4.2).
 *   kind    KLB_D2Q9 (requires nz == 1) or KLB_D3Q19.
 *   geom    SLAB: `width` fluid rows centred in y, `shell` solid rows on each
 *           side, void beyond; walls normal to y; periodic in z.
 *           PIPE: axis at (ny/2, nz/2); a cell centre (y+1/2, z+1/2) at
 *           distance r is fluid if r < radius, solid if radius <= r <
 *           radius + shell, void otherwise.
 *           MASK: `mask` gives the cross-section (host, ny*nz bytes, index
 *           y + ny*z; 0 void, 1 fluid, 2 solid), copied at creation;
 *           periodic_y / periodic_z select periodic cross-section axes.
 *   tau_*   BGK relaxation times of water, electrons, phonons (> 1/2).
 *   rho0    rest density of every species (> 0).
 *   G       uniform body-force density on the water: the pressure drive of
 *           Eq. 2, applied with Guo forcing.
 *   storage KLB_FP64 or KLB_FP32 populations, arithmetic in the same type;
 *           or KLB_FP16_DEV / KLB_BF16_DEV: populations stored in 16 bits as
 *           differences from a per-row FP32 reference population (the row's
 *           x-average, refreshed every 32 steps; FP16 differences scaled by
 *           2^20), FP32 arithmetic, FP64 observables.
 *   iface_bc  KLB_IFACE_SPECULAR (free slip at the liquid/solid interface
 *           for all species, Sec. 4.2) or KLB_IFACE_BOUNCEBACK (the Sec. 4.2
 *           alternative); outer solid faces always bounce back.
 *   phonon_eq KLB_PHONON_FLUID (0, the default: the phonons relax to the
 *           same second-order equilibrium as the other species) or
 *           KLB_PHONON_WAVE: phonons as the linear waves of Sec. 3.4, whose
 *           density obeys the damped wave equation
 *             d_tt n_p - cs^2 d_xx n_p = -gamma_p d_t n_p
 *           (gamma_p = gamma_pC + gamma_pe (1 - u_e/u_p), the friction rates
 *           set by klb_set_couplings).  The phonon equilibrium is then linear
 *           in the momentum, g^eq_i = w_i [drho + 3 c_i . rho u] (moments
 *           drho, rho u and cs^2 drho I: no convective flux), and its forcing
 *           term keeps only (1 - omega/2) w_i 3 c_i . F.  Any other value is
 *           KLB_EINVAL.
 */
typedef struct {
    int32_t kind;
    int32_t nx, ny, nz;
    int32_t geom;
    int32_t width;  /* SLAB */
    int32_t radius; /* PIPE */
    int32_t shell;  /* SLAB, PIPE */
    int32_t periodic_y, periodic_z; /* MASK */
    const uint8_t *mask;            /* MASK */
    double tau_w, tau_e, tau_p;
    double rho0;
    double G[3];
    int32_t storage;
    int32_t iface_bc;
    int32_t phonon_eq;
} klb_desc;

/*
 * Friction coefficients (Eq. 27: F_kl = -F_lk = gamma_kl (u_k - u_l)), as
 * force densities per unit velocity difference, symmetric in k, l:
 *   g_we, g_wp  water-electron and water-phonon, per fluid/solid face
 *               (Eq. 5, Eq. 11, Eq. 15);
 *   g_ep        electron-phonon, per solid cell (Eqs. 12, 15);
 *   g_ec, g_pc  electron and phonon loss to the crystal (Eqs. 13, 16).
 * Negative values (negative quantum friction, Sec. 2) are accepted within the
 * stability bound checked by klb_set_couplings.
 */
typedef struct {
    double g_we, g_wp, g_ep, g_ec, g_pc;
} klb_couplings;

/*
 * Observables of the current step n (after n completed steps): the
 * velocities u(n) of the next step's moment pass.
 *   flow_rate      (1/nx) * sum over fluid cells of u_x.
 *   fit_A, fit_B   least squares u_x = A + B d^2 over fluid cells at distance
 *                  d from the centre plane (slab) / axis (pipe) with
 *                  d_wall - d >= 4; NaN for MASK geometries.
 *   d_wall         slab: width/2; pipe: sqrt(fluid cells per slice / pi).
 *   u_slip         A + B d_wall^2;  dudn_wall = |2 B d_wall|;
 *   slip_length    u_slip / dudn_wall  (L_s = u_s / (du/dy)_w, Sec. 1).
 *   u_wallrow_mean mean u_x over fluid cells with a solid face neighbour.
 *   mean_u[s]      mean u_x of species s over its cells.
 *   momentum[s]    sum of rho u_x;  mass[s] = sum of (rho - rho0).
 *   residual       max over all species cells of |u_x(n) - u_x(n-1)|; NaN
 *                  until two steps have run since creation, init or
 *                  klb_set_state.
 *   nonfinite      number of non-finite density/velocity values.
 *   clipped        16-bit storage: number of species-cells holding a
 *                  population at the largest finite 16-bit magnitude.  The
 *                  encode saturates instead of overflowing to infinity: a
 *                  stored difference (g - ref) * scale beyond +-65504 (FP16,
 *                  scale 2^20: |g - ref| >= 65504 * 2^-20 = 0.0625, ref the
 *                  row's x-average of that population) or +-3.39e38 (BF16,
 *                  scale 1) is written as that bound.  Always 0 for FP32 and
 *                  FP64 storage.
 * All sums are accumulated in FP64 on the device.
 */
typedef struct {
    int64_t step;
    double flow_rate;
    double fit_A, fit_B, d_wall;
    double u_slip, dudn_wall, slip_length;
    double u_wallrow_mean;
    double mean_u[3];
    double momentum[3];
    double mass[3];
    double residual;
    int64_t nonfinite;
    int64_t clipped;
} klb_obs;

/* Device bytes klb_create_lattice needs for this description (0 if the
 * description is invalid): the three population sets of Sec. 4 (two
 * buffers each), the lagged interface velocities of Eq. 27 and small
 * tables.  Pure host computation.  Index widths bound a
 * lattice: the box's cell count nx*ny*nz below 2^32, one direction plane
 * of a species class (its rows x nx padded to 32) below 2^31 elements, and
 * the interface velocities of a class (3 or 6 x its interface rows x padded
 * nx) below 2^31; a class's whole population buffer may exceed 2^31
 * elements (a single lattice can fill the device). */
size_t klb_lattice_bytes(const klb_desc *desc);

/* Sizes of a lattice, from the description alone (host computation; the
 * geometry rules of Sec. 4.2, the nanotube of Sec. 5.1):
 *   fluid_cs / solid_cs     fluid / solid cells of one cross-section;
 *   species_cells[s]        cells carrying species s (whole box);
 *   active_sites            fluid + solid cells (whole box);
 *   iface_cs[2]             fluid / solid cross-section cells with at least
 *                           one fluid/solid face;
 *   max_faces[2]            most such faces of one fluid / solid cell;
 *   d_wall                  wall position of the slip fit (NaN for MASK);
 *   bytes                   klb_lattice_bytes(desc). */
typedef struct {
    int64_t fluid_cs, solid_cs;
    int64_t species_cells[3];
    int64_t active_sites;
    int64_t iface_cs[2];
    int32_t max_faces[2];
    double d_wall;
    uint64_t bytes;
} klb_info;

/* Fill *info for a description; KLB_EINVAL (message via
 * klb_last_error(NULL)) if it is invalid. */
klb_status klb_lattice_info(const klb_desc *desc, klb_info *info);

/*
 * Build the lattice of Sec. 4 (water on the fluid cells, electrons and
 * phonons on the solid cells, Sec. 3.1-3.4) in the caller's device buffer `dev_buf` (at least
 * klb_lattice_bytes(desc) bytes, 256-byte aligned, on the current device)
 * and start from rest: every population deviation and lagged velocity is 0.
 * `cuda_stream` is a cudaStream_t (NULL: the legacy default stream) on which
 * all later work of the handle is enqueued.  `dev_buf` must outlive the
 * handle.  Synchronises the stream once.  Returns KLB_EINVAL for a bad
 * description (tau <= 1/2, rho0 <= 0, non-finite values, nz != 1 for D2Q9, a
 * shell of 0, an empty species, a box beyond the index widths of
 * klb_lattice_bytes),
 * KLB_ENOMEM if `bytes` is too small.  Couplings start at zero.
 */
klb_status klb_create_lattice(const klb_desc *desc, void *dev_buf, size_t bytes,
                              void *cuda_stream, klb_lattice **out);

/* Set the friction coefficients (Eq. 27; Eqs. 5, 11-16).  KLB_EINVAL for non-finite values or for
 * couplings beyond the stability bound of the lagged interface exchange:
 * max over cells of (sum over its faces of |g| of its species pairs) must be
 * below 0.6 rho0 (the two-step-averaged exchange of one face pair is stable
 * for kappa = g (1/rho_k + 1/rho_l) < 4/3, with a margin for density
 * deviations).  Host only; takes effect at the next step. */
klb_status klb_set_couplings(klb_lattice *lat, const klb_couplings *c);

/* Index checks of debug builds (no counterpart in the paper; they stand in
 * for a memory checker).  A library compiled with -DKLB_BOUNDS=1
 * (klb_bounds_checked() returns 1) checks, in every kernel that reads a row
 * record, that the row, its source offsets, the thread's x positions and the
 * interface slots index inside their arrays before anything is touched; a
 * thread that fails records a site code (1 row, 2 source offset, 3 x,
 * 4 slot, 5 partner slot, 6 face count) and skips its cells.
 * klb_bounds_status returns the first recorded site of the lattice (0: none)
 * and clears it; synchronises.  Normal builds never record anything. */
klb_status klb_bounds_status(klb_lattice *lat, uint32_t *site);
int klb_bounds_checked(void);

/* Thermal fluctuations of the water (Eq. 6, the classical
 * fluctuation-dissipation relation of the momentum flux; Eq. 17, its
 * lattice source), in the standard fluctuating lattice Boltzmann form:
 * after each collision the water populations of every fluid cell receive
 *   xi_i = A (a_i - w_i sum_j a_j - 3 w_i c_i . sum_j c_j a_j),
 *   a_i = sqrt(w_i) z_i,  A = sqrt(3 rho0 kT omega_w (2 - omega_w)),
 * with z_i standard normals (Box-Muller) from the Philox-4x32-10
 * counter-based generator keyed by `seed`, counter (x + nx (y + ny z),
 * step mod 2^32, step / 2^32, block of four words).  The noise carries no
 * mass or momentum; the lattice fluid then holds rho0 <u_a^2> = kT.
 * Electrons and phonons are not thermalised.  kT = 0 switches the noise
 * off.  KLB_EINVAL for a negative or non-finite kT, or kT > 0 with 16-bit
 * storage.  Host only; takes effect at the next step.  A lattice with noise
 * cannot join a batch. */
klb_status klb_set_fluctuations(klb_lattice *lat, double kT, uint64_t seed);

/* Start from the local equilibrium (Sec. 4: the second-order polynomial
 * equilibrium of every species, in deviation form) of host fields in box layout:
 * drho[3][ncell] density deviations and u[3][3][ncell] velocities (either
 * may be NULL for zero).  The lagged interface velocities are set to u.
 * Resets the step counter to 0.  Synchronises the stream. */
klb_status klb_init_equilibrium(klb_lattice *lat, const double *drho, const double *u);

/* Advance nsteps >= 0 lattice steps of Sec. 4 (pull streaming with the
 * boundary rules of Sec. 4.2, BGK collision with the drive of Eq. 2 by Guo
 * forcing, interface friction of Eq. 27 from lagged velocities, co-located
 * electron-phonon friction and crystal sinks of Eqs. 12-16) for all three
 * species, one fused kernel per step.  Asynchronous. */
klb_status klb_step(klb_lattice *lat, int64_t nsteps);

/* Compute the observables of the current step into *out (host): the slip
 * length L_s = u_s / (du/dy)_w of Sec. 1 from a fit of the water profile,
 * the flow rate, and the species means, masses and momenta (FP64 sums).
 * Synchronises the stream.  Returns KLB_EUNSTABLE (with *out filled) when a
 * non-finite value was seen, else KLB_ERANGE (with *out filled) when a 16-bit
 * population was stored saturated (out->clipped > 0): the state is then no
 * longer the scheme's. */
klb_status klb_observables(klb_lattice *lat, klb_obs *out);

/*
 * Allocation-free variant of klb_observables().  The paper has no
 * counterpart: this is a service for callers that cannot allocate device
 * memory.  Typical ones embed the library in a host application that owns
 * the device allocator (a fixed pool, or a process running under a hard
 * device-memory cap) and hands out the lattice buffer once; they cannot ask
 * for more, and may want the lattice buffer to hold nothing but the solver
 * state while observations run.
 *
 * Same inputs and output as klb_observables() (the lattice state is read, the
 * observables are written to *out on the host).  The per-block FP64 partial
 * sums and the final sums live in a static device array of this library
 * instead of the lattice buffer: KLB_STATIC_MAX_BLOCKS blocks of 19 doubles
 * plus 32 doubles (about 7.5 MB), held on every GPU that loads the library
 * until the process exits.  Nothing is allocated: no cudaMalloc, cudaFree or
 * allocating library routine is called.
 *
 * - Lattices whose observation pass needs more than KLB_STATIC_MAX_BLOCKS
 *   thread blocks (per cross-section cell, one per 256 x positions with
 *   FP32 arithmetic, one per 128 with FP64 storage) are rejected with
 *   KLB_EINVAL and a message naming the limit.
 * - The first call on a device looks up the device address of the array
 *   (once per device, with that device current); make that first call before
 *   any stream capture.
 * - Every call shares the one array and it keeps the last call's contents.
 *   Each call overwrites every entry it reads, so nothing needs clearing, but
 *   calls that overlap on the GPU (other streams, other host threads, other
 *   lattices) race on it: serialise them.
 * Synchronises the lattice's stream.
 */
#define KLB_STATIC_MAX_BLOCKS 49152
klb_status klb_observables_static(klb_lattice *lat, klb_obs *out);

/* Density deviations drho[3][ncell] and velocities u[3][3][ncell] (the
 * moments of Sec. 4, with the half-force correction of the Guo velocity) of
 * the current step, host, box layout (either may be NULL).  Synchronises. */
klb_status klb_get_field(klb_lattice *lat, double *drho, double *u);

/* Checkpoints (no counterpart in the paper).  Current state to host, box layout: post-collision deviations
 * g[3][Q][ncell] and the velocities of the two previous steps
 * U1[3][3][ncell] = u(n-1), U2 = u(n-2).  The lagged velocities are kept
 * only at interface cells; other cells read 0.  Any pointer may be NULL.
 * Synchronises. */
klb_status klb_get_state(klb_lattice *lat, double *g, double *U1, double *U2);

/* Replace the state (same layouts as klb_get_state; U1/U2 are read at
 * interface cells only) and set the step counter.  Synchronises. */
klb_status klb_set_state(klb_lattice *lat, const double *g, const double *U1,
                         const double *U2, int64_t step);

/*
 * Batches (no counterpart in the paper; they serve design sweeps in the
 * shape of the nanotube study of Sec. 5.1): many independent lattices
 * stepped together, one kernel launch per lattice step for all of them
 * (channels of different sizes and parameters).  All members share the lattice kind, the storage
 * type and the CUDA stream; they may stand at different time levels (a
 * request admitted while others run).  A member's step pattern (state buffer
 * parity, lagged-velocity ring slot and, for 16-bit storage, reference
 * generation and refresh) repeats after 6 steps, or 384 with 16-bit storage,
 * so one table of per-lattice kernel arguments per phase of that period
 * describes every step.  The
 * tables live in the caller's device buffer (klb_batch_bytes), with a count
 * of the periods completed since they were built (the step number each
 * replayed step needs: FP32 storage draws the dither of its fix-up from the
 * cell and the step); a whole period is captured once in a CUDA graph and
 * replayed.  The batch enqueues
 * its work on a stream of its own, ordered after and before the members'
 * stream with events.  Members stay usable on their own between batch calls
 * (observables, fields, state); stepping a member alone takes it out of phase
 * and the next batch call fails with KLB_ESTATE.
 */
typedef struct klb_batch klb_batch;

/* Device bytes a batch of these members needs (0 if they cannot form one). */
size_t klb_batch_bytes(klb_lattice *const *members, int n);

/* Form a batch in the caller's device buffer (256-byte aligned, at least
 * klb_batch_bytes).  The members must outlive the batch.  KLB_EINVAL if they
 * differ in kind, storage or stream, or one appears twice; KLB_ENOMEM if the
 * buffer is too small. */
klb_status klb_batch_create(klb_lattice *const *members, int n, void *dev_buf, size_t bytes,
                            klb_batch **out);

/* Advance every member by nsteps >= 0 steps.  Asynchronous on the members'
 * stream. */
klb_status klb_batch_step(klb_batch *b, int64_t nsteps);

/* Time steps_per_candidate >= 1 steps of the batch with each block width
 * (32, 64 and 128 consecutive x per thread block) and keep the fastest; the
 * timed steps are real steps of the members.  *width (may be NULL) receives
 * the chosen width.  Synchronises. */
klb_status klb_batch_autotune(klb_batch *b, int steps_per_candidate, int *width);

/* Block width in use (128 unless autotuned) and total blocks per step. */
int klb_batch_width(const klb_batch *b);
int64_t klb_batch_blocks(const klb_batch *b);

/* Release the batch (not its members or buffer).  Synchronises. */
klb_status klb_batch_destroy(klb_batch *b);

/* Message of the last failing call on the batch ("" if none). */
const char *klb_batch_last_error(const klb_batch *b);

/*
 * Serving: a request loop for design-sweep solves (no counterpart in the
 * paper, which runs no simulations).  Requests (a lattice description, its
 * couplings, a residual tolerance and limits) may be submitted at any time.
 * The server keeps admitted lattices resident in one caller-provided device
 * arena, admits queued requests first come first served as arena space and
 * member slots free up (a request waits while the one ahead of it does not
 * fit), advances every resident lattice together as one batch, and retires
 * each when its residual (klb_obs.residual) is at most its tolerance, or it
 * reaches its step or time limit, or turns non-finite.
 *
 * klb_server_tick runs one scheduling round: retirement checks of every
 * resident lattice, admissions, re-forming of the batch when its membership
 * changed (with an optional block-width autotune whose steps count as part
 * of the round), then `check_every` steps of the batch.  Every resident
 * lattice therefore advances by exactly check_every steps per round and is
 * checked at multiples of check_every steps since its admission, so a
 * request's result (steps, observables) does not depend on which other
 * requests shared the GPU with it.  Times are seconds on the server's
 * monotonic host clock (klb_server_clock).  Not thread-safe.
 */
typedef struct klb_server klb_server;

typedef struct {
    int32_t kind;          /* lattice kind of every request                  */
    int32_t storage;       /* storage of every request                       */
    int32_t check_every;   /* steps per round (>= 1)                         */
    int32_t max_resident;  /* most lattices resident at once (>= 1)          */
    int32_t autotune_steps;/* > 0: when the batch is re-formed, time 3
                              candidate block widths over this many steps
                              each (plus one warm-up) inside the round;
                              needs check_every >= 3 (autotune_steps + 1)     */
    int32_t pad;
} klb_server_opts;

typedef struct {
    klb_desc desc;         /* MASK cross-sections are copied at submission */
    klb_couplings couplings;
    double tol;            /* retire when residual <= tol (> 0)            */
    int64_t max_steps;     /* step limit (> 0), KLB_ETIMEOUT when reached  */
    double max_seconds;    /* limit on time since arrival (0: none)        */
    double arrival;        /* arrival time (server clock); < 0: now        */
    int64_t id;            /* caller's tag, returned in the result         */
} klb_request;

typedef struct {
    int64_t id;
    int32_t status;        /* KLB_OK converged; KLB_ETIMEOUT step or time
                              limit; KLB_EUNSTABLE non-finite values; other
                              codes if creation failed on the device        */
    int32_t pad;
    int64_t steps;         /* steps run                                    */
    int64_t sites;         /* active sites (fluid + solid cells)           */
    uint64_t bytes;        /* arena bytes held                             */
    double arrival, admitted, finished;  /* server clock                 */
    klb_obs obs;           /* observables at retirement                    */
} klb_result;

typedef struct {
    int64_t queued, resident, finished;
    int64_t rounds, batch_forms;
    uint64_t arena_bytes, bytes_in_use, peak_bytes_in_use, table_bytes;
    double site_updates;   /* sum over rounds of resident sites x steps      */
    int32_t width;         /* block width of the current batch (0: none)    */
    int32_t pad;
} klb_server_stats;

/* Device bytes reserved in the arena for batch argument tables of up to
 * max_resident lattices of this storage. */
size_t klb_server_table_bytes(int storage, int max_resident);

/* Create a server over the caller's device arena (256-byte aligned,
 * larger than klb_server_table_bytes) on `stream` (NULL: legacy default
 * stream).  The arena stays owned by the caller and must outlive the
 * server.  KLB_EINVAL for bad options. */
klb_status klb_server_create(void *arena, size_t arena_bytes, void *stream,
                             const klb_server_opts *opts, klb_server **out);

/* Queue a request.  KLB_EINVAL for an invalid description, couplings or
 * limits, a kind or storage other than the server's, or a lattice that could
 * never fit in the arena (nothing is queued then). */
klb_status klb_server_submit(klb_server *srv, const klb_request *req);

/* One scheduling round (see above).  Synchronises.  *n_finished (may be
 * NULL) receives the number of results now waiting in klb_server_poll. */
klb_status klb_server_tick(klb_server *srv, int64_t *n_finished);

/* Move up to max finished results, oldest first, into out; returns the
 * number moved. */
int64_t klb_server_poll(klb_server *srv, klb_result *out, int64_t max);

/* Counters and the server clock. */
klb_status klb_server_get_stats(const klb_server *srv, klb_server_stats *st);
double klb_server_clock(const klb_server *srv);

/* Release the server and every resident lattice (not the arena); queued
 * requests are dropped.  Synchronises. */
klb_status klb_server_destroy(klb_server *srv);

/* Message of the last failing call on the server ("" if none); a message
 * for a failed creation when srv is NULL. */
const char *klb_server_last_error(const klb_server *srv);

/* Number of completed steps, lattice sizes and species-cell counts
 * (bookkeeping, no counterpart in the paper). */
int64_t klb_get_step(const klb_lattice *lat);
int64_t klb_species_cells(const klb_lattice *lat, int species);

/* Release the handle (not the caller's buffer).  Synchronises.  No
 * counterpart in the paper, as for the error messages below. */
klb_status klb_destroy(klb_lattice *lat);

/* Message of the last failing call on `lat` ("" if none); a message for
 * failures that produced no handle when `lat` is NULL.  Valid until the next
 * call on the same handle. */
const char *klb_last_error(const klb_lattice *lat);

#ifdef __cplusplus
}
#endif

#endif /* KLB_H */
