/*
 * gbpic -- electrostatic PIC-MCC particle cycle on a cell-based adaptive quadtree, for
 * NVIDIA GB300 (sm_103a).  C ABI.
 *
 * The method is that of Kolobov & Arslanbekov, "Electrostatic PIC with adaptive Cartesian
 * mesh" (arXiv:1604.07713):
 *   - §3   : ES-PIC with Monte Carlo collisions of electrons and ions with neutrals, a
 *            multigrid Poisson solver with the potential at cell centres, NGP charge
 *            assignment at cell centres, bilinear interpolation of E from cell corners;
 *            explicit scheme (dx < ~3 Debye lengths, dt < 1/omega_pe).
 *   - §3.1 : one quad-tree grid for motion and collisions; cell-based particle lists (a
 *            particle crossing a face leaves its cell's list and joins the neighbour's);
 *            refinement hands particles to children by position, coarsening to the parent;
 *            statistics reset when the grid changes.
 *   - §2.1 : Morton-ordered cells of a forest of root boxes.
 *   - §4.3 : particle splitting (one particle -> four in 2D) and merging for exponential
 *            growth of electrons and ions in ionization events; the AMR grid as particle
 *            management.
 *
 * Conventions for every call:
 *   - The library owns all device memory.  Host pointers passed in are read during the call
 *     and not kept; host pointers passed out are written during the call.
 *   - No C++ exception crosses this ABI.  Every call returns a pic_status; on failure
 *     pic_last_error() returns a thread-local message.
 *   - A CUDA failure returns PIC_ECUDA and poisons the context: every later call on it
 *     returns PIC_ESTATE (except pic_destroy).
 *   - Read-out calls take a capacity `cap` (elements) and report the required size in
 *     *n_out; when cap is too small they return PIC_EINVAL and write nothing.
 *   - Work is issued on the context's stream (pic_set_stream; default: the legacy default
 *     stream).  Calls that return host data synchronise that stream.
 *   - Units are SI (or any consistent normalised set: eps0, q, m, qe are parameters).
 */
#ifndef GBPIC_H
#define GBPIC_H

#include <stdint.h>

#if defined(__GNUC__)
#define GBPIC_API __attribute__((visibility("default")))
#else
#define GBPIC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pic_ctx pic_ctx; /* opaque, library-owned */

typedef enum {
    PIC_OK = 0,
    PIC_EINVAL = 1,         /* bad argument, size or state for this call */
    PIC_ENOMEM = 2,         /* device or host allocation failed */
    PIC_ECUDA = 3,          /* CUDA runtime error; context poisoned */
    PIC_ESTATE = 4,         /* context poisoned by an earlier error, or call out of order */
    PIC_ECAPACITY = 5,      /* particle population exceeds the configured hard capacity */
    PIC_ETIMEOUT = 6,       /* a bounded device-side wait gave up */
    PIC_ENOTCONV = 7,       /* Poisson solve did not reach mg_rel_tol in mg_max_cycles */
    PIC_WARN_STABILITY = 8  /* explicit-PIC limits of §3 exceeded (dx > 3 lambda_D or
                               omega_pe dt > 1); the call still did its work */
} pic_status;

enum { PIC_FP32 = 0, PIC_FP64 = 1 };
enum { PIC_BC_PERIODIC = 0, PIC_BC_DIRICHLET = 1, PIC_BC_NEUMANN = 2 };
enum { PIC_ADAPT_MESH = 1, PIC_ADAPT_PARTICLES = 2 };
/* Particle shapes (§3): NGP charge assignment at cell centres with the bilinear gather of the
 * corner field (any mesh); on a uniform mesh (max_level 0) also the cloud-in-cell variants
 * CIC-EM (momentum conserving: E at cell centres by central differences, gathered with the
 * deposit's bilinear weights) and CIC-EC (energy conserving: E = -grad of the bilinear
 * interpolant of phi over cell centres).  Beyond a non-periodic wall a cloud's share folds
 * into the boundary cell; phi beyond it takes the Poisson operator's ghost value. */
enum { PIC_SHAPE_NGP = 0, PIC_SHAPE_CIC_EM = 1, PIC_SHAPE_CIC_EC = 2 };

/* Fields per leaf, in leaf (Morton key) order, for pic_read_fields. */
enum {
    PIC_FIELD_PHI = 0,     /* potential at the leaf centre [V] (1 per leaf)                   */
    PIC_FIELD_RHO = 1,     /* charge density, NGP deposit + background [C/m^3] (1 per leaf)   */
    PIC_FIELD_COUNT_E = 2, /* particles of species 0 in the leaf (1 per leaf)                 */
    PIC_FIELD_COUNT_I = 3, /* particles of species 1 in the leaf (1 per leaf)                 */
    PIC_FIELD_NODE_E = 4,  /* E at the leaf's 4 corners (x0,y0),(x1,y0),(x0,y1),(x1,y1),
                              (Ex,Ey) each: 8 per leaf [V/m]                                */
    PIC_FIELD_EMAG = 5,    /* |E| at the leaf centre from the face gradients (1 per leaf)     */
    /* time averages over the steps since the diagnostics were last reset (pic_diag_enable;
       0 when none were taken): */
    PIC_FIELD_AVG_NE = 6,  /* electron density [m^-3]                                         */
    PIC_FIELD_AVG_NI = 7,  /* ion density [m^-3]                                              */
    PIC_FIELD_AVG_TE = 8,  /* electron temperature (2/3) <eps> [eV], 0 where no electrons     */
    PIC_FIELD_AVG_PHI = 9  /* potential [V]                                                   */
};

/* Phases timed by pic_get_timing (CUDA events on the context's stream). */
enum {
    PIC_PHASE_DEPOSIT = 0, PIC_PHASE_POISSON = 1, PIC_PHASE_NODE_E = 2,
    PIC_PHASE_LISTS = 3,        /* per step before the push: list ranks, fill and flag reset */
    PIC_PHASE_SCAN = 4, PIC_PHASE_MOVE = 5, PIC_PHASE_SORT = 6, PIC_PHASE_ADAPT = 7,
    PIC_PHASE_SPLIT_MERGE = 8,
    PIC_PHASE_GRAPH = 9,        /* whole steps of an ensemble replayed as one CUDA graph */
    PIC_N_PHASES = 10
};

/* Plain old data, copied at pic_create.  Species 0 is electrons (elastic + ionization
 * collisions), species 1 ions (elastic collisions with a Maxwellian neutral partner). */
typedef struct pic_config {
    int32_t precision;          /* PIC_FP32 | PIC_FP64: particle state and push arithmetic */
    int32_t n_species;          /* 1 (electrons on a fixed background) or 2               */
    uint64_t seed;              /* Philox key                                              */
    double dt;                  /* time step [s]                                           */
    double eps0;                /* permittivity                                            */
    double q[2], m[2];          /* charge and mass per species                             */
    double qe;                  /* elementary charge: converts J <-> eV in the MCC         */
    int32_t mcc;                /* 0: no collisions                                        */
    int32_t bc_x, bc_y;         /* PIC_BC_*: walls absorb particles unless periodic        */
    int32_t max_level;          /* deepest refinement level below the root boxes (<= 8)    */
    double gas_density;         /* neutral density [m^-3]                                  */
    double gas_temperature_ev;  /* neutral temperature [eV]                                */
    double neutral_mass;        /* neutral mass [kg]                                       */
    double sigma_el;            /* elastic cross section [m^2] (electrons and ions)        */
    double sigma_iz0;           /* ionization: sigma = sigma_iz0 (1 - eps_th/eps), eps>th  */
    double eps_th_ev;           /* ionization threshold [eV]                               */
    double phi_left_dc, phi_left_amp, phi_left_freq; /* x = 0 wall: dc + amp sin(2 pi f t) */
    double phi_right;           /* x = Lx wall potential                                   */
    double rho_background;      /* uniform background charge density                       */
    int32_t ppc_target, ppc_min, ppc_max; /* split/merge band (§4.3): e.g. 32, 8, 128        */
    int32_t adapt_every;        /* informational: steps between pic_adapt calls            */
    double e_ref;               /* reference field for the refinement criterion [V/m]     */
    double refine_field;        /* refine where |E| > refine_field * e_ref                 */
    double coarsen_field;       /* coarsen only where |E| < coarsen_field * e_ref          */
    int32_t refine_count;       /* refine where the electron count exceeds this           */
    int32_t coarsen_count;      /* coarsen 4 siblings whose electron count is <= this      */
    double mg_rel_tol;          /* Poisson: stop at ||b - A phi|| <= tol ||b||              */
    int32_t mg_max_cycles;      /* Poisson: V-cycle limit per solve                        */
    int32_t instance;           /* instance id mixed into the Philox counter               */
    int64_t particle_capacity;  /* per species; 0 = automatic (grows as needed)            */
    int32_t shape;              /* PIC_SHAPE_*: charge assignment and field gather (§3)    */
    int32_t implicit;           /* 1: the direct implicit scheme (§3 DIPIC, NGP shape only):
                                   a predictor drift, the field of the predicted charge with
                                   the susceptibility 1 + (omega_p dt)^2 in the Poisson
                                   operator, then the corrector and the collisions; 0: leapfrog */
} pic_config;

/* Create a context of n_instances independent PIC instances, one config each (cfg points
 * to n_instances structs): the ES-PIC with MCC of electrons and ions with neutrals of §3 (its
 * physical parameters: charges, masses, time step, neutral gas, the analytic cross sections,
 * wall potentials), the refinement and particle-management parameters of §3.1 and §4.3, and
 * the multigrid tolerance of §3.  The device is the current CUDA device.  *out receives the
 * context.  Errors: PIC_EINVAL (bad config), PIC_ENOMEM, PIC_ECUDA. */
GBPIC_API pic_status pic_create(const pic_config *cfg, int32_t n_instances, pic_ctx **out);

/* Release every resource of the context.  NULL is accepted. */
GBPIC_API pic_status pic_destroy(pic_ctx *ctx);

/* Issue all later work on `stream` (a cudaStream_t; NULL = legacy default stream). */
GBPIC_API pic_status pic_set_stream(pic_ctx *ctx, void *stream);

/* Set the leaf mesh of instance `inst` (§2.1 forest of nx0 x ny0 root boxes of side h0
 * with Morton-ordered quadtrees, §3.1).  Leaf i is the cell at refinement level level[i]
 * (0 = root) of root box root[i] (row-major: root = rx + ry * nx0) with Morton code
 * morton[i] inside that root at that level (x in the even bits).  Leaves may come in any
 * order; they must tile the domain and be 2:1 balanced across faces.  root == NULL
 * means the uniform level-0 mesh (n_leaves must equal nx0 * ny0; morton, level ignored).
 * Discards any particles of the instance.  Errors: PIC_EINVAL (not a balanced tiling,
 * level > max_level, sizes), PIC_ENOMEM, PIC_ECUDA. */
GBPIC_API pic_status pic_set_mesh(pic_ctx *ctx, int32_t inst, int32_t nx0, int32_t ny0, double h0,
                        int64_t n_leaves, const uint32_t *root, const uint32_t *morton,
                        const uint8_t *level);

/* Replace the population of species `species` in instance `inst` by n particles given as
 * host arrays of absolute positions x, y, velocities vx, vy, vz and weights w (real
 * particles per macro-particle per unit depth).  id == NULL assigns ids next_id ..
 * next_id + n - 1.  Particles are located in their leaf (half-open cells, floor rule) and
 * put into the leaf's cell-based list (§3.1): by leaf, load order inside a leaf.  After
 * loading species 0 (the electrons) the explicit-PIC limits of §3 are checked as by
 * pic_check_stability: when a leaf is wider than 3 Debye lengths or omega_pe dt > 1 the
 * call returns PIC_WARN_STABILITY (the particles are loaded; pic_last_error() gives the
 * numbers).  Errors: PIC_EINVAL (position outside the domain, id >= 2^32, mesh not set),
 * PIC_ENOMEM, PIC_ECUDA. */
GBPIC_API pic_status pic_load_particles(pic_ctx *ctx, int32_t inst, int32_t species, int64_t n,
                              const double *x, const double *y, const double *vx,
                              const double *vy, const double *vz, const double *w,
                              const uint64_t *id);

/* Advance every instance by n_steps steps of the particle cycle (§3): NGP deposit ->
 * multigrid Poisson -> corner E -> fused gather, leapfrog push, wall handling, leaf
 * location and MCC with electron-ion pair spawning -> cell-list update.  Asynchronous
 * except for capacity checks.  Errors: PIC_ECAPACITY, PIC_ENOTCONV (the step still
 * completed with the last iterate; also when the residual is not finite -- NaN or Inf in the
 * charge density or the potential -- which pic_last_error() names), PIC_ECUDA. */
GBPIC_API pic_status pic_step(pic_ctx *ctx, int32_t n_steps);

/* Compute deposit -> Poisson -> corner E for the current state without moving particles
 * (the field half of a step; pic_step does this itself). */
GBPIC_API pic_status pic_compute_fields(pic_ctx *ctx);

/* Mesh adaptation and particle management (§3.1, §4.3) on every instance.
 * PIC_ADAPT_MESH: refine leaves with more than refine_count electrons or
 * |E| > refine_field e_ref (level < max_level); coarsen sibling quartets with <=
 * coarsen_count electrons and |E| < coarsen_field e_ref; restore 2:1 balance (refinement
 * wins); hand particles to children by position / to the parent; carry phi over.
 * PIC_ADAPT_PARTICLES: per leaf and species, split particles 1 -> 4 while the count is
 * below ppc_min; merge pairs down to ppc_target when it is above ppc_max. */
GBPIC_API pic_status pic_adapt(pic_ctx *ctx, int32_t flags);

/* Copy a per-leaf field (PIC_FIELD_*) of instance `inst` to host memory `out`, in leaf (Morton
 * key) order: the potential at cell centres and the NGP charge density of §3, the per-leaf
 * counts of the cell-based lists of §3.1, the corner field that §3's bilinear gather reads,
 * and the centre |E| of the refinement criterion.  out must hold 8 values per leaf for
 * PIC_FIELD_NODE_E, 1 otherwise; `cap` and `n_out` as in the conventions above.  Fields are
 * those of the last step or pic_compute_fields.  Errors: PIC_EINVAL (unknown field, cap too
 * small, mesh not set), PIC_ECUDA. */
GBPIC_API pic_status pic_read_fields(pic_ctx *ctx, int32_t inst, int32_t field, double *out,
                           int64_t cap, int64_t *n_out);

/* Copy the leaf mesh of instance `inst` (Morton key order) to host arrays; any pointer may
 * be NULL.  root/morton/level as in pic_set_mesh. */
GBPIC_API pic_status pic_read_mesh(pic_ctx *ctx, int32_t inst, uint32_t *root, uint32_t *morton,
                         uint8_t *level, int64_t cap, int64_t *n_out);

/* Copy the population of one species in cell-list order to host arrays (absolute positions,
 * FP64); leaf receives each particle's leaf index.  Any pointer may be NULL. */
GBPIC_API pic_status pic_read_particles(pic_ctx *ctx, int32_t inst, int32_t species, double *x,
                              double *y, double *vx, double *vy, double *vz, double *w,
                              uint64_t *id, uint32_t *leaf, int64_t cap, int64_t *n_out);

/* Population sizes and the last Poisson solve of instance `inst` (any pointer may be NULL):
 * n_leaves, particles of species 0 and 1, V-cycles and final relative residual. */
GBPIC_API pic_status pic_get_counts(pic_ctx *ctx, int32_t inst, int64_t *n_leaves, int64_t *n_e,
                          int64_t *n_i, int32_t *mg_cycles, double *mg_rel_res);

/* Step counter (Philox counter word and RF phase t = step * dt) and next particle id. */
GBPIC_API pic_status pic_get_step(const pic_ctx *ctx, int64_t *step);
GBPIC_API pic_status pic_set_step(pic_ctx *ctx, int64_t step);

/* Per-phase device timing with CUDA events on the context's stream.  pic_set_timing(1)
 * starts recording (clearing earlier records); pic_get_timing synchronises the stream and
 * writes, per phase (PIC_PHASE_*), the summed milliseconds to ms[] and the number of
 * kernel launches to launches[] (either may be NULL), for min(n, PIC_N_PHASES) phases. */
GBPIC_API pic_status pic_set_timing(pic_ctx *ctx, int32_t on);
GBPIC_API pic_status pic_get_timing(pic_ctx *ctx, double *ms, int64_t *launches, int32_t n);

/* Total kernel launches issued by the context since creation. */
GBPIC_API pic_status pic_get_launch_count(const pic_ctx *ctx, int64_t *launches);

/* Cell-list bookkeeping of one species (§3.1 list update; no counterpart in the paper's
 * numbers).  Each leaf's list keeps free slots for particles that enter it during a step.
 * A leaf that receives more entering particles than it has free slots moves to a fresh
 * segment at the tail of the species' buffer (`tail_moves` counts these moves); when the
 * tail is used up, every list of the species is laid out again with fresh free slots
 * (`relayouts` counts the steps that needed it).  `overflowed` = entering records that
 * found no free slot.  All three count since the species was last loaded.  Any pointer may
 * be null.  Synchronizes the context's stream.  Errors: PIC_EINVAL (bad instance or
 * species). */
GBPIC_API pic_status pic_get_list_stats(pic_ctx *ctx, int32_t inst, int32_t species, int64_t *relayouts,
                                        int64_t *tail_moves, int64_t *overflowed);

/* |E| at the leaf centres of instance `inst`, exactly as pic_read_fields(PIC_FIELD_EMAG), for
 * callers that cannot allocate device memory: code whose device memory is fully owned by an
 * outside allocator or a fixed budget (where a cudaMalloc behind its back could fail or break
 * its accounting), and real-time loops that allocate nothing after start-up (cudaMalloc and
 * cudaFree can stall or synchronize the device).  The paper has no counterpart; this is an
 * interface convenience.  It uses a fixed 1 MiB file-scope device array (held by every GPU
 * that loads the library until the process exits) instead of a temporary buffer, so it
 * accepts meshes of at most 131,072 leaves and returns PIC_EINVAL with a message for larger
 * ones.  The first call on a device looks up that array's device address (once per device,
 * with the device current); make that first call before any stream capture.  The current
 * device must be the context's device (else PIC_EINVAL, the context stays usable).  All
 * calls share the one array and it keeps the last call's values: calls that overlap on the
 * GPU (other streams, threads or contexts at the same time) race on it.  `out`, `cap`,
 * `n_out` and the errors are as in pic_read_fields; the call synchronises the stream. */
GBPIC_API pic_status pic_read_emag_noalloc(pic_ctx *ctx, int32_t inst, double *out, int64_t cap,
                                           int64_t *n_out);

/* Launch-shape autotuner (no counterpart in the paper: the launch shapes are this
 * implementation's).  Runs up to max_steps ordinary steps of every instance (they advance the
 * simulation exactly as pic_step does: no result depends on a launch shape), two steps per
 * candidate configuration, times each step with CUDA events on the context's stream and keeps
 * the fastest configuration (a candidate replaces the best one only when at least 2 % faster)
 * for the context's later steps.  The candidates, searched
 * one coordinate at a time: the push kernel's block size (128 or 256 threads) and its
 * resident blocks per SM; for an ensemble whose steps replay as one CUDA graph, also the
 * share of the GPU each instance's push takes inside the graph (1, 1/2, 1/4, 1/8) and the
 * number of parallel graph branches (8, 16, 32).  *steps_used (may be NULL) receives the
 * steps run (at most max_steps; fewer when the candidates or the steps run out).  Status as
 * pic_step. */
GBPIC_API pic_status pic_autotune(pic_ctx *ctx, int32_t max_steps, int32_t *steps_used);

/* The configuration the autotuner chose (or the defaults: 256 threads, all resident blocks,
 * graph share 1/4, 16 branches), and the best step time it measured (0 if never tuned).
 * Any pointer may be NULL. */
GBPIC_API pic_status pic_get_tuning(const pic_ctx *ctx, int32_t *push_threads, int32_t *push_blocks_per_sm,
                                    int32_t *graph_push_div, int32_t *graph_branches, double *best_ms);

/* Time-averaged diagnostics of instance `inst` (§3.3: the discharge results are RF-cycle
 * averages of n_e, n_i, T_e, phi and the electron energy distribution; §3.1: statistics
 * counters are reset when the grid changes).  With n_bins > 0, every later step adds, after its
 * field solve, the stored state (x^n, v^{n-1/2}) and the step's potential to per-leaf sums of
 * the electron and ion weights, the electrons' weighted kinetic energy eps = m |v|^2 / (2 qe)
 * [eV] and phi, and the weight of every electron inside region = {x0, x1, y0, y1} (absolute,
 * [x0, x1) x [y0, y1); NULL = the whole domain) to an energy histogram of n_bins (<= 512)
 * bins of width eps_max_ev / n_bins (energies >= eps_max_ev are not binned).  The sums are
 * reset by this call, by pic_diag_reset and by every mesh change (pic_adapt with
 * PIC_ADAPT_MESH, pic_set_mesh).  n_bins = 0 turns the diagnostics off.  Read them with
 * pic_read_fields (PIC_FIELD_AVG_*) and pic_read_eedf.  Every sum is taken in a fixed order:
 * two runs give the same bits.  Instances with diagnostics on are stepped without the
 * ensemble's captured graph.  Errors: PIC_EINVAL (n_bins > 512, eps_max_ev <= 0). */
GBPIC_API pic_status pic_diag_enable(pic_ctx *ctx, int32_t inst, int32_t n_bins, double eps_max_ev,
                                     const double *region);
GBPIC_API pic_status pic_diag_reset(pic_ctx *ctx, int32_t inst);

/* The electron energy distribution of the diagnostics' region accumulated since the reset,
 * normalised as a density in energy: f[b] = S_b / (sum_b S_b * d_eps) [1/eV] for the bin
 * [b d_eps, (b + 1) d_eps), S_b the summed weights (all 0 when nothing was binned).
 * *samples (may be NULL) receives the steps accumulated.  cap / n_out as for read-outs
 * (n_bins values).  Errors: PIC_EINVAL (diagnostics off, cap too small). */
GBPIC_API pic_status pic_read_eedf(pic_ctx *ctx, int32_t inst, double *f, int64_t cap, int64_t *n_out,
                                   int64_t *samples);

/* The explicit-PIC limits of §3 (cells smaller than about 3 Debye lengths, omega_pe dt < 1)
 * for given plasma parameters: n_e_max the largest electron density over leaves [m^-3],
 * w_leaf_max the largest electron weight sum of a leaf (n_e h^2 per unit depth [m^-1]),
 * t_e_ev the electron temperature [eV], with q[0], m[0], eps0, qe and dt of *cfg.  Writes
 * max h / lambda_D = sqrt(w_leaf_max q^2 / (eps0 kT)) (infinite when kT = 0 and electrons
 * are present) and max omega_pe dt = sqrt(n_e_max q^2 / (eps0 m)) dt (either pointer may be
 * NULL).  Returns PIC_WARN_STABILITY when the first exceeds 3 or the second 1, else PIC_OK.
 * A host computation: needs no context and no GPU.  Errors: PIC_EINVAL (negative inputs,
 * non-positive eps0, m[0] or qe). */
GBPIC_API pic_status pic_stability_limits(const pic_config *cfg, double n_e_max, double w_leaf_max, double t_e_ev,
                                          double *dx_over_debye, double *wpe_dt);

/* The same limits for the current electron population (species 0) of instance `inst`: per
 * leaf the weight sum and density from the cell lists, the temperature from the weighted
 * velocity variance of the whole population (kT = m <|v - <v>|^2> / 3).  Writes the two
 * ratios and T_e [eV] (any pointer may be NULL); returns PIC_WARN_STABILITY or PIC_OK as
 * pic_stability_limits.  Synchronises the stream.  Errors: PIC_EINVAL (mesh not set),
 * PIC_ECUDA. */
GBPIC_API pic_status pic_check_stability(pic_ctx *ctx, int32_t inst, double *dx_over_debye, double *wpe_dt,
                                         double *t_e_ev);

/* Checkpoint of instance `inst` (no counterpart in the paper): a self-contained byte image of
 * every piece of state the following steps read -- the leaf mesh, the potential with the
 * previous solution and the solve count of the multigrid warm start, the wall potentials of
 * the last solve, the context's step counter and the instance's next particle id, and per
 * species the cell lists (records in list order, in the state's precision) with the per-leaf
 * weight sums left for the next deposit.  Writes the image to `buf` (host memory of `cap`
 * bytes) and its size to *bytes; with buf == NULL or cap too small it only reports the size
 * and returns PIC_EINVAL.  Synchronises the stream.  Errors: PIC_EINVAL, PIC_ECUDA. */
GBPIC_API pic_status pic_checkpoint_write(pic_ctx *ctx, int32_t inst, void *buf, int64_t cap, int64_t *bytes);

/* Restore instance `inst` from an image of pic_checkpoint_write taken from an instance of the
 * same configuration (precision, species, max_level must match; the image is checked).  The
 * mesh and both populations are replaced and the context's step counter is set to the
 * image's.  Later steps and adaptations then give bit for bit the results the checkpointed
 * run gives.  Errors: PIC_EINVAL (not an image of this version, configuration mismatch,
 * truncated), PIC_ECAPACITY, PIC_ENOMEM, PIC_ECUDA. */
GBPIC_API pic_status pic_checkpoint_read(pic_ctx *ctx, int32_t inst, const void *buf, int64_t bytes);

/* Host-side fault injection for tests of the failure paths (no counterpart in the paper; no
 * GPU fault is made).  PIC_FAULT_ALLOC: after `count` more device allocations from the
 * context's block cache (every mesh, particle and temporary buffer), the next one fails as a
 * failed cudaMalloc would, and the call that made it returns PIC_ENOMEM (the context stays
 * usable).  PIC_FAULT_BALANCE: pic_adapt's 2:1 balance closure gives up after `count`
 * sweeps (1..64; normally 64) with PIC_ETIMEOUT, before the mesh is changed.
 * PIC_FAULT_NONE clears both.  Errors: PIC_EINVAL. */
enum { PIC_FAULT_NONE = 0, PIC_FAULT_ALLOC = 1, PIC_FAULT_BALANCE = 2 };
GBPIC_API pic_status pic_inject_fault(pic_ctx *ctx, int32_t kind, int64_t count);

/* Thread-local message of the last failing call on this thread ("" if none). */
GBPIC_API const char *pic_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* GBPIC_H */
