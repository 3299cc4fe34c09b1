/*
 * dem.h -- C ABI of the GB300 (sm_103a) DEM hot path for the adaptive
 * coarse-grain method of Queteschiner, Lichtenegger, Schneiderbauer and Pirker,
 * "Adaptive Coarse-Graining for Large-Scale DEM Simulations" (CFD 2017).
 *
 * What a step computes (one call of dem_step advances every instance of a
 * context by one time step per count):
 *   - contact forces of the non-linear damped Hertzian spring-dashpot model,
 *     normal part Eq. 3, tangential part Eq. 4 with a per-contact tangential
 *     overlap carried over the contact's life, Coulomb truncation Eq. 5,
 *     coefficients k_n, gamma_n, k_t, gamma_t and beta(e) of Eq. 6
 *     (Sec. 2.1), plus gravity and an optional moving floor plane;
 *   - Newton's equations for translation and rotation (Eqs. 1-2), advanced by
 *     velocity Verlet with the two half kicks of consecutive steps merged;
 *   - cell-list neighbour lists, rebuilt on the device whenever the
 *     accumulated displacement bound reaches half the skin.  The paper names
 *     neighbour-list rebuilds as a cost driver (Sec. 3, runtimes) but
 *     describes no search; the design here is this library's own.
 *
 * Conventions shared by all calls:
 *   - Units are SI.  Particle arrays are float64, concatenated over the
 *     context's instances in instance order; within an instance particles
 *     are in ID order (ID = index of the particle in the array written by
 *     dem_write, 0 .. n_k - 1).  Vectors are row-major (n, 3).
 *   - Device state is float32 (velocities, angular velocities, masses,
 *     forces) and 32-bit fixed point for positions and radii: a length is
 *     an integer multiple of the instance's quantum q = 2^k m, the smallest
 *     power of two with (largest box extent) / q <= 2^30.  Written
 *     positions and radii are rounded to the nearest multiple of q;
 *     positions read back are exact multiples of q.
 *   - Memory: every device byte the library uses is the caller's workspace
 *     (size from dem_query_workspace), passed to dem_create and owned by the
 *     caller until dem_destroy.  The library never allocates or frees device
 *     memory and never frees caller memory.
 *   - Streams: all work is ordered on the stream given to dem_create; calls
 *     return before the GPU work completes unless stated otherwise.  A host
 *     pointer (any pointer that cudaPointerGetAttributes does not report as
 *     device or managed memory) makes dem_read/dem_write stage through the
 *     workspace and synchronise the stream before returning.
 *   - Errors: host-detectable errors return at once and leave the context
 *     unchanged.  Errors found on the device (list overflow, non-finite
 *     force, escaped particle) set a device status word; dem_sync_status
 *     reads it, and once set every later call returns that status.  No
 *     kernel traps or aborts.  dem_last_error gives a one-line message.
 */
#ifndef DEM_H
#define DEM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dem_ctx dem_ctx;

typedef enum {
    DEM_OK = 0,
    DEM_ERR_ARG = 1,        /* invalid argument or configuration */
    DEM_ERR_CAPACITY = 2,   /* neighbour-list width or particle capacity exceeded */
    DEM_ERR_CUDA = 3,       /* a CUDA runtime call failed */
    DEM_ERR_NONFINITE = 4,  /* a force, torque or velocity became NaN/Inf */
    DEM_ERR_ESCAPED = 5,    /* a particle left the representable z range */
    DEM_ERR_TIMEOUT = 6,    /* a bounded device wait gave up */
    DEM_ERR_STATE = 7,      /* call not valid in the context's current state */
    DEM_ERR_BOUNDS = 8      /* (library built with DEM_CHECKS=1 only) a gathered particle index of the
                               step kernel, or a cell code or candidate range of the list build, out
                               of range; the access was skipped */
} dem_status;

/* Fields of dem_read / dem_write.  n counts particles. */
typedef enum {
    DEM_F_POS = 0,      /* (n,3) float64 position [m]; read/write */
    DEM_F_VEL = 1,      /* (n,3) float64 velocity at the current integer step [m/s]; read/write */
    DEM_F_OMEGA = 2,    /* (n,3) float64 angular velocity [1/s]; read/write */
    DEM_F_RADIUS = 3,   /* (n)   float64 radius [m]; read/write */
    DEM_F_MASS = 4,     /* (n)   float64 mass [kg]; read/write (write after RADIUS) */
    DEM_F_FORCE = 5,    /* (n,3) float64 total force at the current step [N]; read only */
    DEM_F_TORQUE = 6,   /* (n,3) float64 total torque at the current step [N m]; read only */
    DEM_F_WALL_XI = 7,  /* (n,3) float64 tangential overlap of the floor contact [m] (0 if none); read, and
                           write after the state and the contacts to resume a run (stored as float32; kept if
                           the particle touches the floor at the next evaluation) */
    DEM_F_NBR_COUNT = 8,/* (n)   float64 neighbour-list length of each particle; read only */
    DEM_F_FEXT = 9      /* (n,3) float64 external force held on each particle [N], added to the contact and
                           gravity forces every step until overwritten (written by the coupling controllers,
                           or by the caller; stored as float32) */
} dem_field;

/* One independent DEM system ("instance").  A context advances all of its
 * instances together; every instance has its own box, material and count. */
typedef struct {
    int64_t n;            /* particles written by dem_write (IDs 0 .. n-1) */
    int64_t capacity;     /* maximum particles (>= n) */
    double lo[3], hi[3];  /* box; periodic axes wrap on [lo, hi), z is open above */
    int32_t periodic[3];  /* x and y may be periodic; z must not be */
    int32_t floor_on;     /* 1: frictional floor plane at z = lo[2] */
    double floor_v[3];    /* floor velocity [m/s] (tangential part acts through friction) */
    double g[3];          /* gravity [m/s^2] */
    double dt;            /* time step [s] */
    double skin;          /* neighbour-list skin [m] */
    double r_max;         /* largest radius that will ever be present [m] */
    double E, nu, e, mu;  /* Young's modulus [Pa], Poisson ratio, restitution, friction (Eq. 6) */
    double mu_wall;       /* particle-wall friction; < 0 means use mu */
    double rho;           /* particle density [kg/m^3]; masses default to rho 4/3 pi r^3 */
    int32_t clamp_fn;     /* 1: drop tensile normal forces (not in Eq. 3; default 0) */
    int32_t reserved;
} dem_instance_desc;

typedef struct {
    int32_t n_instances;              /* >= 1 */
    int32_t max_neighbors;            /* list width L_max, 1 .. 32 */
    const dem_instance_desc *inst;    /* n_instances descriptors (host memory) */
} dem_config;

typedef struct {
    double q;            /* length quantum [m] */
    double lo[3], hi[3]; /* box as represented (hi - lo is a multiple of q) */
    int32_t ncell[3];    /* cell grid */
    int32_t reserved;
    int64_t n;           /* current particle count */
    int64_t capacity;
} dem_instance_info;

typedef struct {
    int64_t steps;           /* steps taken since dem_create */
    int64_t rebuilds;        /* neighbour-list builds (all instances) */
    int64_t list_entries;    /* sum of list lengths at the last dem_stats call */
    int64_t contacts;        /* contacts (particle pairs counted from both sides + floor) at that call */
    int64_t particles;       /* live particles */
    int64_t wall_contacts;   /* floor contacts among `contacts` */
    int32_t step_threads;    /* threads per block of the step kernel in use (dem_set_step_block) */
    int32_t step_lanes;      /* lanes per particle of the step kernel (dem_set_step_lanes) */
    int32_t graph_fused;     /* 1: the captured graph runs fused steps (dem_set_graph_mode) */
    int32_t reserved;
} dem_stats_t;

/* Bytes of device workspace a context with this configuration needs. */
dem_status dem_query_workspace(const dem_config *cfg, int64_t *bytes_out);

/* Create a context on the current CUDA device.  workspace: device pointer,
 * 256-byte aligned, >= dem_query_workspace bytes, owned by the caller.
 * stream: cudaStream_t (NULL = legacy default stream).  The state is
 * undefined until POS, VEL, OMEGA and RADIUS have been written. */
dem_status dem_create(const dem_config *cfg, void *workspace, int64_t workspace_bytes,
                      void *stream, dem_ctx **out);

/* Release the context (not the workspace).  Synchronises the stream. */
dem_status dem_destroy(dem_ctx *ctx);

/* Write a field for all particles (n = sum of the instances' counts).
 * Writing POS, VEL, OMEGA, RADIUS or MASS starts the system afresh from this
 * state: contact histories are cleared, the neighbour lists rebuilt and the
 * first step begins with a half kick from the forces at this state. */
dem_status dem_write(dem_ctx *ctx, int32_t field, const void *src, int64_t n);

/* Read a field at the current integer step.  VEL, OMEGA, FORCE, TORQUE and
 * WALL_XI evaluate the contact forces at the current state (no state change). */
dem_status dem_read(dem_ctx *ctx, int32_t field, void *dst, int64_t n);

/* Contacts at the current step, per particle in ID order: partner IDs
 * (ascending, -1 padded; width entries per particle) of the particles it
 * overlaps, and the tangential overlap xi (Eq. 4) of each such contact, in
 * the frame of the pair's lower ID (xi of pair (a, b) with a < b is the same
 * vector in both rows).  partner: int32 (n, width); xi: float64 (n, width, 3).
 * Single-instance contexts only. */
dem_status dem_read_contacts(dem_ctx *ctx, int32_t *partner, double *xi, int32_t width, int64_t n);

/* The neighbour lists the next step walks, per particle in ID order: the partner IDs of
 * every entry of its row (ascending, -1 padded; width entries per particle): the pairs within
 * r_i + r_j + skin at the last list build, and those of particles inserted since (Sec. 2.3
 * insertion adds rows without a list build).  A pending list build runs first.  partner:
 * int32 (n, width), device memory; more entries than width: DEM_ERR_CAPACITY at the next
 * status check.  Single-instance contexts only.  Not in the paper: for inspection and tests. */
dem_status dem_read_neighbors(dem_ctx *ctx, int32_t *partner, int32_t width, int64_t n);

/* Set tangential overlaps of existing neighbour pairs (same layout as
 * dem_read_contacts); pairs not within the neighbour skin are ignored.  Use
 * after dem_write to resume a run; the lists are built first if needed. */
dem_status dem_write_contacts(dem_ctx *ctx, const int32_t *partner, const double *xi, int32_t width,
                              int64_t n);

/* Advance nsteps time steps (asynchronous). */
dem_status dem_step(dem_ctx *ctx, int64_t nsteps);

/* Synchronise the stream and return the device status word as a dem_status. */
dem_status dem_sync_status(dem_ctx *ctx);

/* Per-instance description of the represented system. */
dem_status dem_instance_info_get(dem_ctx *ctx, int32_t instance, dem_instance_info *out);

/* Counters (synchronises). */
dem_status dem_stats(dem_ctx *ctx, dem_stats_t *out);

/* Capture dem_step in CUDA graphs of `steps_per_graph` steps (0 disables).
 * The neighbour-list rebuild sits in a conditional node set by the step
 * kernel, so a captured run needs no host round trip. */
dem_status dem_set_graph(dem_ctx *ctx, int32_t steps_per_graph);

/* Threads per block of the step kernel (the fused force and integration of Eqs. 1-6):
 * 0 (automatic, the default), 64, 128, 256 or 896; anything else is DEM_ERR_ARG.  896 is one
 * block per SM whose warps claim the slices of a contiguous range of tiles in order (single-
 * instance contexts only, else DEM_ERR_STATE); automatic takes it for a single instance with
 * one lane per particle and at least a tile for every resident 128-thread block, else 128.
 * Results do not depend on it (every particle sums its own row in row order); it changes how
 * the work is spread over the GPU.  A captured graph is rebuilt with it.  Not in the paper: a
 * tuning parameter of this implementation.  DEM_ERR_STATE for a block other than 0 or 128
 * threads while more than one lane per particle is set. */
dem_status dem_set_step_block(dem_ctx *ctx, int32_t threads);

/* Lanes per particle of the step kernel: 1 (the default), 2, 4 or 8, or 0 to choose by size
 * (one lane while the context's slots fill half the GPU's resident threads of the one-lane
 * kernel, else the most lanes whose threads are all resident at once; one lane unless the
 * block is 128 threads); anything else is DEM_ERR_ARG, and more than one needs the 128-thread
 * block (DEM_ERR_STATE otherwise).  With
 * L lanes, lane l of a particle's group evaluates the contacts of its row entries l, l + L,
 * l + 2L, ... (Eqs. 3-6) and the group adds its partial force and torque sums in a fixed
 * order before the first lane integrates (Eqs. 1-2): for systems too small to fill the GPU
 * with one thread per particle.  Results are deterministic for a given L (they do not depend
 * on the block size or the schedule) and differ between values of L only by the order of the
 * float sums.  A captured graph is rebuilt with it.  Not in the paper: a tuning parameter of
 * this implementation. */
dem_status dem_set_step_lanes(dem_ctx *ctx, int32_t lanes);

/* How a captured graph (dem_set_graph) runs its steps.  1: one step-kernel launch per step,
 * each preceded by a conditional list-build node.  2: fused steps: one cooperative launch
 * (one block per 128-slot tile, or as many blocks as are resident at once, each walking a
 * range of tiles) runs every step up to the next list build, with a grid barrier
 * between steps (the last block to arrive ends the step for every instance); the graph loops
 * (a conditional while node) over list build + fused launch until its steps are done.  Each
 * step computes exactly what the per-step kernel computes (the same bits); fused steps save
 * the per-step launch and node latency of systems too small to fill the GPU.  Needs one lane
 * per particle and 128-thread blocks (DEM_ERR_STATE otherwise; the previous graph is kept).
 * 0 (the default): fused when those hold and a block for every 128-slot tile holding live
 * particles is resident at once, else one launch per step.  A barrier wait that does not end within about a second reports
 * DEM_ERR_TIMEOUT.  With fused steps dem_graph_step_kernel_ms times the whole graph launch
 * (list builds included) and counts its steps.  Not in the paper: a scheduling choice of this
 * implementation. */
dem_status dem_set_graph_mode(dem_ctx *ctx, int32_t mode);

/* How the neighbour lists are built (the cell-range and list-build step of the rebuild; the
 * list is the same either way, bit for bit): 0 (the default), each thread scans the 27 cells around
 * its particle in the cell-ordered positions through the caches; 1, each block first stages
 * the cell-ordered positions around its 64 particles in shared memory and reads the candidates
 * that fall there from it.  DEM_ERR_ARG for other values.  A captured graph is rebuilt with it.
 * Not in the paper: an implementation choice (the staged build measured slower on the 1M bed). */
dem_status dem_set_list_build(dem_ctx *ctx, int32_t staged);

/* For tests of the fused steps' failure path: the next fused launch's first block does not
 * arrive at its first grid barrier and leaves, so the other blocks' bounded waits run out
 * (about a second) and the launch ends with DEM_ERR_TIMEOUT in the status word (read by
 * dem_sync_status); the context keeps the error.  Nothing else sets it; no effect without
 * fused steps.  Not in the paper. */
dem_status dem_test_stall_barrier(dem_ctx *ctx);

/* CUDA-event time of step kernels of the most recent graph launch: every fifth
 * step kernel of the graph (the first, the sixth, ...) is bracketed by event
 * nodes; total_ms = the sum over those, count = their number (total_ms / count is
 * the mean duration of a step kernel).  Synchronises the stream.  DEM_ERR_STATE if
 * no graph was built. */
dem_status dem_graph_step_kernel_ms(dem_ctx *ctx, double *total_ms, int32_t *count);

/* ---------------------------------------------------------------------------
 * Differentiable rollouts (gradients of observables with respect to the
 * material parameters E, e and mu of Eq. 6, per instance).
 *
 * dem_rollout_forward runs nsteps steps with the neighbour lists frozen (built
 * once at the start; if a particle moves more than half the skin the run stops
 * with DEM_ERR_CAPACITY) and saves the full state every checkpoint_every steps
 * in the caller's rollout workspace (device memory, 256-byte aligned, size from
 * dem_rollout_workspace).  dem_rollout_adjoint then computes, by a hand-written
 * reverse pass through the contact law and the integrator, the gradient of
 *     J = sum_k ( w_KE,k KE_k + w_R,k runout_k )
 * at the final step, where KE = sum 1/2 m v^2 + 1/2 I w^2 and runout = the
 * largest horizontal distance of a particle from the instance's axis.  Each
 * checkpointed segment is recomputed forward (bit-identical) and walked
 * backwards; which contacts exist and which slip is taken from that forward
 * pass (the derivative is that of the discrete map with the contact pattern
 * held fixed).  The context ends in the rollout's final state.
 *   weights: host (B, 2) {w_KE, w_R}; axis: host (B, 2) {x, y} [m];
 *   grad: host (B, 3) {dJ/dE, dJ/de, dJ/dmu} (mu also moves the floor friction
 *   when mu_wall was left unset).
 * ------------------------------------------------------------------------- */
dem_status dem_rollout_workspace(dem_ctx *ctx, int64_t nsteps, int64_t checkpoint_every, int64_t *bytes);
dem_status dem_rollout_forward(dem_ctx *ctx, int64_t nsteps, int64_t checkpoint_every, void *workspace,
                               int64_t workspace_bytes);
dem_status dem_rollout_adjoint(dem_ctx *ctx, const double *weights, const double *axis, double *grad);

/* Observables at the current step: out (B, 2) = {KE, runout} with axis (B, 2)
 * as above (host arrays; synchronises). */
dem_status dem_observables(dem_ctx *ctx, const double *axis, double *out);

/* Replace the material parameters {E, e, mu} of every instance (host (B, 3));
 * nu, rho and the state are kept.  mu also sets the floor friction when
 * mu_wall was left unset. */
dem_status dem_set_material(dem_ctx *ctx, const double *params);

/*
 * Neighbour counts without any allocation or workspace.  The paper has no
 * counterpart; this is a service for callers that cannot give the library
 * device memory: a host solver or plugin framework that owns every device
 * byte through its own pool and passes only its particle buffers, or a
 * real-time loop that must not allocate after start-up.
 *
 * For n particles of one box it writes counts[i] = the number of j != i with
 * |x_i - x_j| < r_i + r_j + skin (minimum image on periodic axes), with the
 * positions, radii and skin rounded to the same length quantum and tested by
 * the same exact integer arithmetic as a context built from this box, so the
 * counts equal that context's neighbour-list lengths (DEM_F_NBR_COUNT).
 *   x: device float64 (n,3); r: device float64 (n); counts: device int32 (n),
 *   written asynchronously on `stream` (cudaStream_t, NULL = legacy default).
 *   lo, hi, periodic: host arrays of 3; skin >= 0; r_max >= every r.
 * Limits: n <= 262,144 particles and a cell grid (cell width >= 2 r_max +
 * skin) of at most 262,144 cells; larger inputs return DEM_ERR_CAPACITY with
 * a message in dem_last_error(NULL), before any GPU work.
 * Memory: scratch is one fixed 9 MiB device array inside the library, held by
 * every GPU that loads it until the process exits; nothing is allocated or
 * freed.  Every call looks up that array's device address on the current
 * device (cudaGetSymbolAddress), so a device reset between calls is safe;
 * make the first call on a device before any stream capture (it loads the
 * library's module there).  Particles outside an open axis count as being in
 * its edge cells, like a context's; their counts are exact only inside the
 * box.  All calls share the array and each call
 * re-initialises what it reads, so calls that overlap on the GPU (other
 * streams, other threads, or concurrent contexts on the same device) race
 * and must be serialised by the caller.
 */
dem_status dem_neighbor_counts_noalloc(const double *x, const double *r, int64_t n, const double lo[3],
                                       const double hi[3], const int32_t periodic[3], double skin,
                                       double r_max, int32_t *counts, void *stream);

/* ---------------------------------------------------------------------------
 * Two-way volumetric coupling of a coarse-grain level and an embedded fine
 * level (Sec. 2.3).  Both contexts hold one instance each and share one frame
 * of reference; both advance `interval` steps between calls of dem_couple.
 *
 * Geometry: the fine region is the box [lo, hi].  Each face named in
 * feed_faces (coarse material flows in through it) is divided into square
 * surface cells of side >= surface_cell; behind each surface cell, inside the
 * region, lies one hexahedral transition cell of thickness `layer`.  The
 * region is also divided into cubic correction cells of edge >= corr_cell.
 *
 * One call of dem_couple, in the paper's order:
 *  - measurement on the coarse level: mass of coarse particles whose centre
 *    entered the region through each surface cell since the previous call
 *    (integer multiples of mass_unit), their diameter histogram (`bins` bins
 *    over [0, 2 r_max of the fine level] after division by alpha), and the
 *    Favre (mass-weighted) velocity of coarse particles within one diameter
 *    of the face (Sec. 2.3);
 *  - per transition and correction cell on both levels: volume fraction,
 *    Favre velocity, largest speed, and the granular stress of Eq. 7
 *    (contact part 1/2 r_ij f_ij over contacts, floor and axisymmetric-wall
 *    contacts with the branch vector from the contact point to the centre,
 *    plus m v' v');
 *  - stress PI controller per transition cell on the normal stress along the
 *    face normal (setpoint: coarse, process variable: fine):
 *    e = s_cg - s_fine, I += e T_c, u = kp e + ki I; every fine particle in
 *    the cell receives F = u pi r^2 max(0, 1 - s / (1.5 d)) n_in (s: distance
 *    from the face, n_in: inward normal), shortened so that its speed after one
 *    step stays below the coarse cell's largest speed; held until the next call;
 *  - fine-to-coarse P controller per correction cell: target velocity v* =
 *    fine Favre velocity (mode 0) or that times min(phi_fine / phi_cg, 4)
 *    (mode 1, mass flow); every coarse particle in the cell receives
 *    F = kv m (v* - v_cg) / T_c, held until the next call;
 *  - insertion of fine particles per surface cell by simple sequential
 *    inhibition: until the inserted mass reaches the entered mass plus the
 *    carry of earlier intervals, draw a diameter from the histogram (uniform
 *    within the bin) and a position uniformly in the slab behind the cell
 *    (depth max(d, |v_n| T_c)), reject it if it overlaps any fine particle, an
 *    earlier insertion or one of the fine level's axisymmetric walls, or lies
 *    outside the vessel those walls enclose (dem_set_walls), give up after
 *    max_attempts rejections; inserted
 *    particles take the cell's Favre velocity; random numbers come from the
 *    SplitMix64 generator on counters (seed, cell, interval, attempt, draw);
 *  - fine particles whose centre left the region through a drain face are
 *    removed.  Inserted and removed particles take effect at the fine level's
 *    next list build, which the call requests.  Fine particle IDs are never
 *    reused: inserted particles get new IDs, removed IDs read as NaN.
 * ------------------------------------------------------------------------- */
typedef struct dem_coupler dem_coupler;

typedef struct {
    double lo[3], hi[3];    /* fine region [m] */
    int32_t feed_faces;     /* bit 2a: face at lo[a], bit 2a+1: face at hi[a] */
    int32_t drain_faces;    /* same bits: fine particles past these faces are removed */
    double surface_cell;    /* surface / transition cell side [m] (3 to 10 coarse diameters) */
    double layer;           /* transition layer thickness [m] */
    double corr_cell;       /* correction cell edge [m] */
    int32_t interval;       /* steps between calls (T_c = interval dt) */
    int32_t bins;           /* diameter histogram bins, 1 .. 32 */
    double alpha;           /* coarse diameter / fine diameter */
    double kp, ki;          /* stress PI gains [-], [1/s] */
    double kv;              /* fine-to-coarse P gain [-] */
    int32_t mode;           /* 0: velocity, 1: mass flow */
    int32_t max_attempts;   /* SSI rejections per cell and call before giving up */
    uint64_t seed;          /* random seed of the insertion */
    double mass_unit;       /* unit of the integer mass bookkeeping [kg] */
    int32_t max_insert;     /* most particles inserted per surface cell and call */
    int32_t add_forces;     /* 0: the controller forces replace the levels' held forces; 1: they are added
                               (for a level shared by two couplers; clear with dem_clear_external_force) */
    double velocity_below;  /* with velocity_below_on: correction cells whose centre lies below this
                               height [m] take the velocity target (mode 0) whatever `mode` says: Sec. 3
                               applies a pure velocity coupling to coarse particles that passed the
                               silo's orifice */
    int32_t velocity_below_on;  /* 0 (a zero-initialised spec): velocity_below is ignored */
    int32_t reserved;
} dem_coupling;

typedef enum {
    DEM_CPL_SURFACE_MASS = 0,    /* (S)   mass entered through each surface cell at the last call [kg] */
    DEM_CPL_SURFACE_CARRY = 1,   /* (S)   mass still to insert [kg] */
    DEM_CPL_SURFACE_INSERTED = 2,/* (S)   particles inserted at the last call */
    DEM_CPL_SURFACE_VEL = 3,     /* (S,3) Favre velocity at the face [m/s] */
    DEM_CPL_SURFACE_HIST = 4,    /* (S,bins) diameter histogram of the entered particles */
    DEM_CPL_LAYER_STRESS = 5,    /* (H,2,6) stress {xx,yy,zz,xy,xz,yz} [Pa], coarse then fine */
    DEM_CPL_LAYER_PHI = 6,       /* (H,2) volume fraction */
    DEM_CPL_LAYER_VEL = 7,       /* (H,2,3) Favre velocity */
    DEM_CPL_LAYER_VMAX = 8,      /* (H,2) largest speed */
    DEM_CPL_LAYER_CTRL = 9,      /* (H,3) {error, integral, u} of the stress controller */
    DEM_CPL_CORR_PHI = 10,       /* (C,2) volume fraction, coarse then fine */
    DEM_CPL_CORR_VEL = 11,       /* (C,2,3) Favre velocity */
    DEM_CPL_SIZES = 12           /* (4) {S, H, C, calls so far} */
} dem_coupler_field;

dem_status dem_coupler_workspace(dem_ctx *coarse, dem_ctx *fine, const dem_coupling *spec, int64_t *bytes);
dem_status dem_coupler_create(dem_ctx *coarse, dem_ctx *fine, const dem_coupling *spec, void *workspace,
                              int64_t workspace_bytes, dem_coupler **out);
/* One coupling call, queued on the fine level's stream after the work queued on the coarse
 * level's (an event); the host does not wait.  The device updates the fine level's count;
 * the first later call that needs the count on the host (dem_read, dem_write, dem_counts,
 * dem_instance_info_get, dem_stats, the contact I/O) synchronises to fetch it.  Inserting
 * beyond the fine level's capacity inserts nothing and sets DEM_ERR_CAPACITY, reported at
 * that synchronisation or at dem_sync_status. */
dem_status dem_couple(dem_coupler *cp);
dem_status dem_coupler_read(dem_coupler *cp, int32_t field, double *dst, int64_t n);
/* Free the coupler (not its workspace).  It does not touch the two contexts,
 * which may be destroyed before or after it; call it when no dem_couple of
 * this coupler is running. */
dem_status dem_coupler_destroy(dem_coupler *cp);

/* Zero the held external (coupling) force of every particle of the context. */
dem_status dem_clear_external_force(dem_ctx *ctx);

/* Live particles and IDs handed out, per instance (host arrays of B; synchronises).  Particles
 * marked for removal count as live until a list build drops them: after a coupling call, the
 * next step's; after falling below a removal height, the next build the displacements call
 * for.  Reads return NaN for them at once. */
dem_status dem_counts(dem_ctx *ctx, int64_t *live, int64_t *ids);

/* Volume-averaged fields of instance k on a uniform grid of n[0] x n[1] x n[2] cubic cells of
 * edge h [m] from lo[3] (cell (i, j, l) spans lo + h (i, j, l) .. lo + h (i+1, j+1, l+1)):
 * out (device memory, float64, 5 values per cell, x fastest) = {solid volume fraction
 * (volume of the particles whose centre lies in the cell over the cell volume), mass [kg],
 * mass-weighted (Favre) velocity [m/s] (0 in empty cells)}, at the current step.  The
 * paper evaluates output at any location from the finest level available there (Sec. 2.3);
 * a caller composes that from these per-level grids (levels.py does).  out_len must be
 * 5 n[0] n[1] n[2].  Asynchronous on the context's stream. */
dem_status dem_grid_fields(dem_ctx *ctx, int32_t k, const double lo[3], double h, const int32_t n[3], double *out,
                           int64_t out_len);

/* Axisymmetric walls of instance k, for vessels such as the silo of Sec. 3 (a cone below a
 * cylinder): the surface of revolution of the polyline points[2 i] = rho_i [m] (>= 0),
 * points[2 i + 1] = z_i [m], i < npts, about the vertical axis through (axis[0], axis[1]) [m].
 * Every segment is a wall of its own, end points included (a free rim is an edge contact): a
 * particle touches segment i where its distance to the segment, measured in the particle's
 * own azimuthal half-plane, is below its radius.  Each contact is a particle-wall contact of
 * Eqs. 3-6 (the wall at rest with infinite radius and mass, the particle's material, the wall
 * friction mu_wall) with the normal from the nearest point of the segment to the centre.  A
 * segment from rho = 0 is a disk: (0, z_o) - (r_o, z_o) closes an orifice of radius r_o.
 * npts = 0 removes the walls; otherwise 2 <= npts <= 8 and consecutive points differ.  The
 * tangential overlaps of up to two segment contacts per particle are kept (a third
 * simultaneous one, which needs two kinks within a particle diameter, starts from zero each
 * step); setting the walls clears them.
 * Particles whose centre falls below z_remove [m] at a step are removed at that step (their
 * IDs are not reused; reads return NaN for them): each is parked out of reach of every live
 * particle and dropped at the next list build, which it does not force.  z_remove =
 * -INFINITY (or a height more than about 2^31 length quanta below the box) removes none.
 * Their number and mass accumulate in dem_wall_removed.  The walls and the removal apply to dem_step, graphs and the read-out of
 * velocities and forces; dem_rollout_forward refuses a context that has either
 * (DEM_ERR_STATE).  Synchronises the context's stream. */
dem_status dem_set_walls(dem_ctx *ctx, int32_t k, const double *axis, int32_t npts, const double *points,
                         double z_remove);

/* Particles and mass [kg] removed below z_remove in instance k since the context was
 * created: out[0] = count, out[1] = mass (host array of 2; synchronises). */
dem_status dem_wall_removed(dem_ctx *ctx, int32_t k, double *out);

/* Last error message of the context; with ctx == NULL, the last configuration
 * error (dem_query_workspace / dem_create) of the calling thread.  Never NULL. */
const char *dem_last_error(const dem_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* DEM_H */
