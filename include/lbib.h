/*
 * lbib.h -- C ABI of the GB300 (sm_103a) LB-IB-MLS adhesion solver.
 *
 * The library advances 2D lattice Boltzmann channels (D2Q9 BGK, Eq. 1-6 of
 * Coclite et al., arXiv:1808.01448) coupled to rigid particles through an
 * immersed boundary with moving-least-squares interpolation and spreading
 * (Sec. "The combined LB-IB method"), hydrodynamic loads from probes
 * (Eq. 7-8), stochastic ligand-receptor bonds (Eq. 9-11), a wall force
 * (Eq. 12) and a second-order rigid-body update (Eq. 13-16).  Every step of
 * that path runs in the library's CUDA kernels.
 *
 * Conventions shared by all calls:
 *  - Every call returns an lbib_status and never aborts; on failure
 *    lbib_last_error() gives a message (thread-local, valid until the next
 *    failing call on the same thread).
 *  - Structs are copied at the call; the caller keeps every pointer it
 *    passes.  Array arguments named *_host are host memory.
 *  - The library owns all device memory of a simulation (allocated in
 *    lbib_create / lbib_add_particle / first step, freed in lbib_destroy),
 *    through the caller's allocator hook when one is given.
 *  - Stepping is asynchronous on the configured CUDA stream; read calls
 *    synchronise that stream and the streams of the batches that hold the
 *    simulation, so they see every step enqueued before them.  A
 *    device-side error (a non-finite state, a bounded wait that ran out) is
 *    reported by the next call.
 *  - A handle is not thread-safe; different handles are independent.
 *  - Device waits are bounded: a wait of the lattice pass on its staged
 *    copies gives up after LBIB_WAIT_POLLS polls (environment variable read
 *    when a batch is created; default 65536) and the next call reports
 *    LBIB_E_TIMEOUT.  Calls show as NVTX ranges in profiler timelines.
 *  - Lattice units: dx = dt = 1, c_s^2 = 1/3, nu = (tau - 1/2) / 3.
 *  - Node arrays are row-major [ny][nx]; populations [9][ny][nx] with the
 *    D2Q9 order e_0 = (0,0), e_1..4 = (1,0), (0,1), (-1,0), (0,-1),
 *    e_5..8 = (1,1), (-1,1), (-1,-1), (1,-1) (Eq. 3).
 */
#ifndef LBIB_H
#define LBIB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum lbib_status {
    LBIB_OK = 0,
    LBIB_E_ARG = 1,          /* invalid argument; nothing was changed */
    LBIB_E_OOM = 2,          /* device or host allocation failed */
    LBIB_E_CUDA = 3,         /* a CUDA runtime call failed */
    LBIB_E_STATE = 4,        /* call not allowed in the handle's state */
    LBIB_E_UNSTABLE = 5,     /* the state became non-finite */
    LBIB_E_TIMEOUT = 6,      /* a bounded device wait ran out */
    LBIB_E_UNSUPPORTED = 7,  /* feature not built / not supported by device */
    LBIB_E_BOUNDS = 8        /* a bounds check of the debug build failed */
} lbib_status;

/* Wall kinds for the bottom (y = 0) and top (y = ny - 1) rows.
 * ZOU_HE: known-velocity wall nodes on rows 0 and ny-1 (the paper's walls,
 *         Sec. "The combined LB-IB method", ref. [40]).
 * BOUNCE_BACK: half-way bounce-back, wall lines at y = -1/2 and ny - 1/2,
 *         with the moving-wall correction 6 w_i (e_i . u_w).
 * PERIODIC: both walls periodic (set on both or neither). */
typedef enum lbib_wall { LBIB_WALL_ZOU_HE = 0, LBIB_WALL_BOUNCE_BACK = 1,
                         LBIB_WALL_PERIODIC = 2 } lbib_wall;

/* Storage of the populations in device memory.  Collision arithmetic is
 * FP32 for F32/F16/BF16 and FP64 for F64.  Populations are stored as
 * deviations f_i - w_i; F16 stores them times a power-of-two scale. */
typedef enum lbib_storage { LBIB_STORE_F32 = 0, LBIB_STORE_F64 = 1,
                            LBIB_STORE_F16 = 2, LBIB_STORE_BF16 = 3 } lbib_storage;

/* Rounding of the 16-bit stores (F16, BF16; ignored otherwise).
 * STOCHASTIC (the default): round up with probability equal to the dropped
 * fraction, from a hash of the node index and of the value (the same bits
 * alone or in a batch), so that increments smaller than half a unit in the
 * last place are not lost on average.  NEAREST: round to nearest even; slow
 * transients then stall where the per-step change is below half an ulp. */
typedef enum lbib_rounding { LBIB_ROUND_STOCHASTIC = 0, LBIB_ROUND_NEAREST = 1 } lbib_rounding;

/* Optional device allocator hook (e.g. a framework's caching allocator).
 * alloc returns device memory of at least `bytes` bytes usable on `stream`,
 * or NULL; free releases it.  When NULL the library uses cudaMalloc. */
typedef void *(*lbib_alloc_fn)(size_t bytes, void *stream, void *ctx);
typedef void (*lbib_free_fn)(void *ptr, void *stream, void *ctx);

/* Channel and model parameters (Sec. "Modeling the adhesion dynamics",
 * Table 1).  The physical part mirrors the problem statement:
 *  nx, ny            lattice size (nx >= 8, ny >= 4; nx * ny < 2^31)
 *  wall_bottom/top   lbib_wall
 *  tau               BGK relaxation time (> 1/2), Eq. 1
 *  u_bottom, u_top   tangential wall velocities (x), e.g. u_top = u_max
 *  gx, gy            uniform body-force density (Poiseuille drive, Eq. 4)
 *  k_f, k_r0, kBT    forward / reverse rates per step and thermal energy,
 *                    Eq. 10-11
 *  sigma_star_ratio  sigma* / sigma (0.5: slip bonds), Eq. 11
 *  y_cr, y_eq_ratio  critical bond length and y_cr,eq / y_cr, Eq. 9
 *  hamaker, eps_min  Eq. 12 constant H_k and the lower clamp of the gap
 *  receptor_bottom/top receptor density on each wall (1 = fully covered)
 *  seed, sim_id      key of the counter-based bond draws
 * Device-side settings:
 *  storage           lbib_storage
 *  rounding          lbib_rounding of F16 / BF16 stores
 *  f16_scale         F16 only: power-of-two scale of f - w (0 = automatic)
 *  cuda_stream       cudaStream_t to run on (NULL = the legacy default)
 *  alloc, free, alloc_ctx   optional allocator hook */
typedef struct lbib_config {
    int32_t nx, ny;
    int32_t wall_bottom, wall_top;
    double tau;
    double u_bottom, u_top;
    double gx, gy;
    double k_f, k_r0, kBT;
    double sigma_star_ratio, y_cr, y_eq_ratio;
    double hamaker, eps_min;
    double receptor_bottom, receptor_top;
    uint64_t seed, sim_id;
    int32_t storage;
    int32_t rounding;
    double f16_scale;
    void *cuda_stream;
    lbib_alloc_fn alloc;
    lbib_free_fn free;
    void *alloc_ctx;
    /* Direct-forcing passes per step (multi-direct forcing; 0 or 1: the
     * single pass of Sec. "The combined LB-IB method").  With M > 1 each
     * marker's force is corrected M - 1 times by the slip left after its own
     * particle's force is spread: F <- F + F0 - I[spread(F)], I the MLS
     * interpolation at the marker and F0 the first pass's force; the last F
     * is spread.  0 .. 16, else E_ARG. */
    int32_t ib_iterations;
    /* Spreading scale eps_l of the IB force (Sec. "The combined LB-IB
     * method", MLS transfer of ref. [39]): 0 the element length S_l; 1 the
     * scales solved so that interpolating the spread of a uniform marker
     * force returns it at every marker, sum_m A_lm eps_m = 1 with
     * A_lm = sum_k phi_k(X_l) phi_k(X_m), solved every step at the new
     * pose.  With 1, a particle whose markers closer than 4 sqrt 2 lattice
     * units lie more than LBIB_VB_MAX_BAND apart along its outline (a very
     * thin or small particle) is refused by lbib_add_particle (E_ARG). */
    int32_t ib_spread;
    /* Streaming of the populations: 0 A/B (two buffers, the next step's
     * populations pulled from the last step's), 1 in place (AA pattern: one
     * buffer, so half the population memory; the steps alternate between
     * reading a node's own slots and writing its neighbours' and the
     * reverse).  The same results bit for bit; a batch with an in-place
     * member runs one lattice-pass form (vector loads and stores where the
     * layout allows, no copy-engine variants), so lbib_batch_autotune has
     * nothing to time. */
    int32_t stream_mode;
    int32_t reserved2;
} lbib_config;

/* A rigid particle (Sec. "Pressure and viscous stresses"): a closed polygon
 * of nl linear elements in its body frame (counter-clockwise, centroid at
 * the origin).  When vx/vy are NULL the outline is generated: shape 0 is a
 * circle of radius a, shape 1 an ellipse with semi-axes a (body x) and b
 * (body y), with n_vertices vertices (0 = one per unit of perimeter) at
 * equal arc length.  Pose (xc, yc, theta); density rho_p (mass = rho_p *
 * area); ligand_density is the fraction of elements carrying a ligand,
 * spread evenly; sigma is the spring constant of Eq. 9.  fixed != 0 holds
 * the pose (loads and bonds are still computed).  The outline must fit the
 * on-chip force tile: max radius <= LBIB_MAX_PARTICLE_RADIUS and
 * 3 <= nl <= LBIB_MAX_MARKERS. */
#define LBIB_MAX_MARKERS 512
#define LBIB_VB_MAX_BAND 8
#define LBIB_MAX_PARTICLE_RADIUS 44.0
#define LBIB_MAX_PARTICLES_PER_SIM 16

typedef struct lbib_particle {
    int32_t n_vertices;
    int32_t fixed;
    const double *vx, *vy;
    int32_t shape;
    int32_t reserved0;
    double a, b;
    double xc, yc, theta;
    double rho_p;
    double ligand_density;
    double sigma;
} lbib_particle;

/* Particle state after the last completed step: pose and velocities, the
 * loads of that step (hydrodynamic Eq. 7-8, bond Eq. 9, wall Eq. 12), mass
 * properties, and counts of elements, ligands, probing and bonded ligands.
 * p_adhesion is the probability of adhesion of the paper's Fig. 6 at this
 * step: bonded ligands over the ligands close enough to a receptor wall to
 * bond (n_bonded / n_probing; 0 when none is).  gap_bottom / gap_top: the
 * smallest distance from an element centroid to the bottom / top wall line
 * at the pose of that step's bonds (the paper's separation distance y_min;
 * negative when a centroid lies beyond the wall line; +inf before the first
 * step or with periodic walls), as Eq. 12 takes it before its clamp. */
typedef struct lbib_particle_state {
    double xc, yc, theta, u, v, omega;
    double Fh[2], Mh;
    double Fb[2], Mb;
    double Fw[2];
    double area, mass, inertia, r_eq;
    int32_t nl, n_ligands, n_probing, n_bonded;
    double p_adhesion;
    double gap_bottom, gap_top;
} lbib_particle_state;

typedef struct lbib_state {
    int64_t step;          /* completed steps */
    int32_t n_particles;
    int32_t storage;
    int32_t nx, ny;
} lbib_state;

typedef struct lbib_sim lbib_sim;
typedef struct lbib_batch lbib_batch;

/* Create a simulation; populations start at f = f^eq(rho = 1, u = 0).
 * Errors: E_ARG (invalid config), E_OOM, E_CUDA. */
lbib_status lbib_create(const lbib_config *cfg, lbib_sim **out);

/* Free all memory of the handle (synchronises its stream).  NULL is a no-op. */
lbib_status lbib_destroy(lbib_sim *sim);

/* Add a particle before the first step; *pid receives its index.
 * Errors: E_ARG (bad outline, too large, too many), E_STATE (already
 * stepped), E_OOM. */
lbib_status lbib_add_particle(lbib_sim *sim, const lbib_particle *p, int32_t *pid);

/* Receptor density on a wall (0 bottom, 1 top), before the first step.
 * Bonds form only to walls with density > 0; the forward rate of Eq. 10 is
 * scaled by the density.  Errors: E_ARG, E_STATE. */
lbib_status lbib_set_receptors(lbib_sim *sim, int32_t wall, double density);

/* Set the post-collision populations f*_i of "step -1" ([9][ny][nx], host,
 * full f, not deviations) before the first step.  Page-locked host memory
 * the device can address is read in place by the import kernel; other host
 * memory is copied through a device scratch of 72 bytes per node (kept for
 * later reads).  Returns after the import (the buffer may be reused).
 * Errors: E_STATE, E_CUDA, E_OOM (scratch). */
lbib_status lbib_set_populations(lbib_sim *sim, const double *f_post_host);

/* Enqueue nsteps time steps (weak coupling, Sec. "Fluid-structure
 * interaction strategy"): collide + stream, loads, bonds, wall force, rigid
 * update, IB forcing.  Asynchronous; nsteps == 0 is a no-op.
 * Errors: E_ARG (nsteps < 0), E_CUDA, E_UNSTABLE (reported late). */
lbib_status lbib_step(lbib_sim *sim, int64_t nsteps);

/* Batched stepping: all simulations of a batch advance together, on the
 * first simulation's stream.  Per step, one lattice launch covers the nodes
 * away from the particles of all members (on a second, library-owned
 * stream), one covers the boxes around the particles, and one particle
 * launch runs the loads, bonds, update and IB forcing of every particle; the
 * first overlaps the particle launch of the previous step.  All members must
 * share storage and device.  A simulation may be stepped alone or in a
 * batch, not both concurrently.  lbib_batch_step replays captured CUDA
 * graphs: of 32 steps, then of 4 steps for the rest of the call (each graph
 * captured on its first use and kept until the launch configuration
 * changes), and launches the last 1-3 steps directly. */
lbib_status lbib_batch_create(lbib_sim *const *sims, int32_t n, lbib_batch **out);
lbib_status lbib_batch_step(lbib_batch *b, int64_t nsteps);
lbib_status lbib_batch_destroy(lbib_batch *b);
/* Kernel timing with CUDA events: when nsamples > 0, later batch steps
 * record kernel durations (event records inside the replayed graphs, taken
 * in up to nsamples 32-step graphs in turn, and in the steps a call launches
 * directly): the lattice pass of the middle step of a graph (or of the
 * directly launched steps) and the particle and near-box passes of the step
 * after it.
 * lbib_batch_kernel_times fills mean_ms[3] and count[3] with the
 * mean duration (ms) and number of samples taken since the last call:
 * [0] the lattice pass (the bulk pass when particle work is overlapped),
 * [1] the particle pass, [2] the near-box lattice pass (0 samples when not
 * overlapped).  It synchronises the stream. */
lbib_status lbib_batch_set_timing(lbib_batch *b, int32_t nsamples);
lbib_status lbib_batch_kernel_times(lbib_batch *b, double *mean_ms, int64_t *count);
/* Threads per particle CTA (one element per thread): 512 fits every
 * particle; 256 (FP32 / 16-bit storage, every particle with at most 256
 * elements) holds a quarter of an SM's registers while the particle pass
 * runs, so the bulk lattice pass keeps more of the GPU.  Same results either way.  A
 * new batch takes 256 when it can and has at least 32 particles, else 512.
 * Errors: E_ARG (other widths, or 256 where a particle does not fit). */
lbib_status lbib_batch_set_particle_threads(lbib_batch *b, int32_t threads);
/* Particle states of every member of the batch, in member order (each
 * member's particles in pid order), as lbib_read_state gives them: one
 * gather kernel and one copy to pinned host memory for the whole batch.
 * lbib_batch_read_particles_async only enqueues them on the batch's stream
 * (the states after all work enqueued so far) and returns; the next
 * lbib_batch_read_particles then waits for that copy alone (work enqueued
 * in between keeps running) and converts it.  Without a started readback,
 * lbib_batch_read_particles starts one and waits.  Starting a second one
 * before collecting the first is E_STATE.  out receives up to cap states;
 * *count (if not NULL) the batch's particle count; *d2h_bytes (if not NULL)
 * the bytes copied from the device (the particles' device records and one
 * error word per member).  Reports a member's deferred device error
 * (E_UNSTABLE, E_TIMEOUT) like lbib_read_state. */
lbib_status lbib_batch_read_particles(lbib_batch *b, lbib_particle_state *out, int32_t cap,
                                      int32_t *count, size_t *d2h_bytes);
lbib_status lbib_batch_read_particles_async(lbib_batch *b);
/* Wait for all work enqueued on the batch and report a member's deferred
 * device error (E_UNSTABLE, E_TIMEOUT): one copy of every member's error
 * word.  A started readback stays pending. */
lbib_status lbib_batch_synchronize(lbib_batch *b);
/* Benchmark form of lbib_batch_step: advances the batch nsteps steps with
 * the same results, with the L2 cache flushed before every step, and times
 * the steps alone.  Before each step the library overwrites the caller's
 * device buffer `flush` (flush_bytes bytes; 16-byte aligned, a multiple of
 * 16 bytes and at least the device's L2 size, else LBIB_E_ARG) and, when
 * clean = 1, reads it back, so that the step starts with none of its inputs
 * in L2 and (clean = 1) no dirty line to write back.  The buffer's contents
 * are destroyed.  Steps run as graphs of up to 32 steps, each step joined
 * before the next flush (no overlap between steps).  If ms is not NULL it
 * receives, summed over the steps, the device time (CUDA events) of
 * [0] each step from the end of its flush to the end of its last kernel,
 * [1] its bulk lattice pass, [2] its flush, [3] its near-box and particle
 * passes (the particle pass alone when not overlapped): ms[4].  Synchronises
 * the stream after every graph. */
lbib_status lbib_batch_step_flushed(lbib_batch *b, int64_t nsteps, void *flush,
                                    size_t flush_bytes, int32_t clean, double *ms);
/* Kernel variants of the lattice pass (the bulk pass when particle work is
 * overlapped), all on the same 1024-node tiles: 0 = 256 threads x one
 * group of four nodes; 1 = the same, at most 64 registers (four CTAs per
 * SM); 2 = the same, five CTAs per SM (48 registers); 3 = six CTAs per SM
 * (40 registers);
 * 4 = variant 1 with each plane's source range staged in shared memory by
 * bulk asynchronous copies (copy engine, mbarrier completion); 5 = a
 * pipeline of such copies: eight tiles per CTA through a ring of shared-memory
 * stages (four for 16-bit storage, two for FP32), one producer warp issuing
 * the copies of the next tiles while eight warps compute the current one.
 * Variants 4 and 5 need FP32/FP16/BF16 storage, rows of whole 16-byte words
 * and walls that are not periodic in every member (else they run as
 * variant 1).  FP64 storage and the plain (non-overlapped) pass
 * always use variant 0.  A new batch starts with variant 1.
 * lbib_batch_autotune runs the lattice pass of each variant `reps` times on
 * the batch's current state (timing runs: they write only the buffer the next
 * step overwrites and leave step counters alone, so the simulation is
 * unchanged), keeps the fastest for later steps, writes its index to
 * *variant and the mean milliseconds of each variant to ms[] (either may be
 * NULL).  Synchronises the stream.  lbib_batch_set_variant selects a variant
 * directly (e.g. one tuned on an earlier batch of the same shape). */
#define LBIB_LATTICE_VARIANTS 6
lbib_status lbib_batch_autotune(lbib_batch *b, int32_t reps, int32_t *variant, double *ms);
lbib_status lbib_batch_set_variant(lbib_batch *b, int32_t variant);

/* Nodes each lattice pass of the next step updates, at the particles'
 * current near boxes: nodes[0] the lattice (bulk) pass, nodes[1] the
 * near-box pass (NBx x NBy per particle, rows outside the lattice left out; 0
 * when not overlapped), nodes[2] all nodes of the members.  For the
 * algorithmic bytes of the timed passes.  Synchronises the stream and reads
 * the particle structs back (a few hundred bytes per particle). */
lbib_status lbib_batch_pass_nodes(lbib_batch *b, int64_t *nodes);

/* Wait for all enqueued work of the handle; reports deferred device errors. */
lbib_status lbib_synchronize(lbib_sim *sim);

/* Read the state (synchronises).  Any output may be NULL.  Fields are the
 * density and the velocity u = (sum_i f_i e_i + (g + f_ib)/2) / rho of the
 * current step (Eq. 5-6), each [ny][nx] host doubles; n_nodes must be
 * nx * ny when a field pointer is given.  parts receives up to n_parts
 * particle states. */
lbib_status lbib_read_state(lbib_sim *sim, lbib_state *st, lbib_particle_state *parts,
                            int32_t n_parts, double *rho_host, double *ux_host,
                            double *uy_host, size_t n_nodes);

/* Post-collision populations of the last step (full f, [9][ny][nx]). */
lbib_status lbib_read_populations(lbib_sim *sim, double *f_post_host);

/* Bond state of a particle: bond[l] in {0, 1} and the anchor x of each
 * element's bond (n must equal the particle's element count). */
lbib_status lbib_read_bonds(lbib_sim *sim, int32_t pid, uint8_t *bond_host,
                            double *anchor_x_host, int32_t n);

/* IB force density of the current step on the lattice ([ny][nx] each). */
lbib_status lbib_read_ib_force(lbib_sim *sim, double *fx_host, double *fy_host);

/* Kinematic record of a particle: pose and velocities after the last
 * completed step and one step earlier (the two levels the second-order
 * update of Eq. 13-16 reads), and the particle's completed step count, the
 * counter of its bond draws (Eq. 10-11). */
typedef struct lbib_particle_record {
    double xc, yc, theta, u, v, omega;
    double xc1, yc1, theta1, u1, v1, omega1;
    int64_t step;
} lbib_particle_record;

/* Read a particle's record (synchronises).  Errors: E_ARG, E_CUDA and a
 * deferred device error. */
lbib_status lbib_get_particle_record(lbib_sim *sim, int32_t pid, lbib_particle_record *out);

/* Overwrite a particle's record (synchronises): the next step starts from
 * this pose and history, and the IB forcing of that step is recomputed at
 * the new pose from the current populations (what the end of a step leaves).
 * Bonds and anchors are kept.  Used to prescribe a particle's motion or to
 * replay a trajectory.  Errors: E_ARG (bad pid, non-finite values, negative
 * step), E_CUDA. */
lbib_status lbib_set_particle_record(lbib_sim *sim, int32_t pid, const lbib_particle_record *in);

/* Checkpoints.  A checkpoint is a host blob holding everything later steps
 * depend on: the post-collision populations in the storage format, the
 * completed step count, and per particle its record, last loads and counts,
 * bond flags and anchors.  lbib_checkpoint_size gives its size;
 * lbib_checkpoint_save writes it into host memory of at least that size
 * (synchronises; E_ARG if too small); lbib_checkpoint_load restores it into
 * a simulation created with the same lattice, storage (and F16 scale) and
 * particles added with the same element counts (E_ARG otherwise; nothing is
 * changed then), recomputes the IB forcing of the coming step, and
 * synchronises.  Stepping on from a loaded checkpoint gives the same bits as
 * stepping on from the saved simulation. */
lbib_status lbib_checkpoint_size(lbib_sim *sim, size_t *bytes);
lbib_status lbib_checkpoint_save(lbib_sim *sim, void *host, size_t bytes);
lbib_status lbib_checkpoint_load(lbib_sim *sim, const void *host, size_t bytes);

/* Device memory the simulation holds now (populations, particles, scratch
 * and its own stepping tables), in bytes; for admission control. */
lbib_status lbib_device_bytes(lbib_sim *sim, size_t *bytes);

/* Allocation-free IB forcing (no counterpart in the paper: a service for
 * callers that cannot allocate device memory -- plugins and solvers inside a
 * host application that owns every device allocation through its own arena,
 * and real-time loops that must not call an allocator, which can
 * synchronise the device or fail under memory pressure, once running).
 *
 * Computes the IB force density f_ib of one rigid particle (the MLS direct
 * forcing of lbib_step's first pass, with desired marker velocity
 * (u, v) + omega x (X_l - X_c)) on a lattice given by cfg and its
 * post-collision populations, and writes it to fx_dev, fy_dev.
 *  cfg        channel; storage must be LBIB_STORE_F32; cfg->cuda_stream is
 *             the stream the work is queued on (NULL: legacy default stream);
 *             the allocator fields are ignored
 *  f_dev      device, [9][ny][nx] FP32 deviations f_i - w_i (caller-owned)
 *  p          particle; an explicit outline (vx, vy, n_vertices) is required
 *  fx_dev, fy_dev  device, [ny][nx] doubles (caller-owned), fully written
 * Allocates no device or host heap memory: its only scratch is one static
 * device array of 256 KiB that every GPU loading the library keeps until the
 * process exits.  The first call on a device looks up that array's device
 * address (cudaGetSymbolAddress, once per device) with the device current;
 * make that first call before any stream capture.  The call copies nothing
 * from host memory: it enqueues three kernels on the stream (one writes the
 * descriptors and tables, passed as kernel parameters, into the array) and
 * returns without waiting for them.  Calls share the array and each rewrites
 * what it reads; calls whose work overlaps on the GPU (different streams)
 * race.  Errors: E_ARG (bad arguments, or the particle needs more than the
 * 256 KiB scratch or the shared memory of one SM), E_CUDA, E_UNSUPPORTED
 * (device index >= 64). */
lbib_status lbib_ib_force_noalloc(const lbib_config *cfg, const float *f_dev,
                                  const lbib_particle *p, double u, double v, double omega,
                                  double *fx_dev, double *fy_dev);

const char *lbib_last_error(void);

/* Library build information ("lbib <version> sm_103a ..."). */
const char *lbib_version(void);

#ifdef __cplusplus
}
#endif
#endif
