/*
 * sph.h -- C ABI of the GB300 (sm_103a) SPH-with-boids step library.
 *
 * The library advances the method of "A GPU-based Hydrodynamic Simulator with
 * Boid Interactions" (Liu, Kayar, Perlin, arXiv 2311.15088) by whole steps:
 * uniform-grid binning with a counting sort (sections "Neighborhood Search",
 * "Neighbor Search with Sorting"), poly6 density and the equation of state
 * (sections "Smoothed Particle Hydrodynamics", "Pressure and Viscosity"),
 * symmetrised pressure + viscosity pair forces with the boid-touch counters
 * (section "Pressure and Viscosity", listing "Compute acceleration"), the boid
 * rules with two-way coupling (section "Boid Motion and Agent Fluid
 * Interaction") and Euler-Cromer integration with damped walls (section
 * "Governing Equations" frame loop, section "Background").
 *
 * Conventions shared by every entry point:
 *   - Return value: SPH_OK (0) or one of the SPH_ERR_* codes; the message of
 *     the last failure is sph_last_error(handle) (or sph_last_error(NULL)
 *     for failures before a handle exists).
 *   - Pointers are device pointers unless an `on_host` argument says
 *     otherwise.  Host pointers given with on_host = 1 should be pinned for
 *     asynchronous copies; the call then synchronises `stream` before it
 *     returns so that the host buffer is complete.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default).
 *   - The caller owns every buffer, including the workspace; the library
 *     never allocates or frees device memory.  sph_destroy frees only the
 *     host-side handle.
 *   - float4 arrays are (x, y, z, w) with w ignored on input and 0 on output.
 *   - Particle ids: ids 0 .. n_boid-1 are the particles attached to boids
 *     (boid b <-> particle b), ids n_boid .. n_boid+n_fluid-1 are the fluid
 *     particles (fluid index f <-> id n_boid + f), as the paper's
 *     initialize_particle kernel assigns them.
 *   - No entry point falls back to the CPU.
 */
#ifndef SPH_GB300_H
#define SPH_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define SPH_OK           0
#define SPH_ERR_ARG      1  /* invalid parameter, size, pointer or alignment   */
#define SPH_ERR_CUDA     2  /* a CUDA runtime call or launch failed            */
#define SPH_ERR_OVERFLOW 3  /* a size does not fit the library's index types   */
#define SPH_ERR_TIMEOUT  4  /* a bounded device wait gave up                   */
#define SPH_ERR_STATE    5  /* call out of order (e.g. fields before a step)   */

/* Constant sets of the spiky-gradient / viscosity-Laplacian prefactors. */
#define SPH_MULLER3D      0  /* 45/(pi h^5) for both: the 3-D normalised kernels (default) */
#define SPH_PAPER_LITERAL 1  /* 30/(pi h^4) and 40/(pi h^4), as printed in the paper      */

/* Fluid -> boid coupling modes. */
#define SPH_COUPLE_FORCE 0   /* v_b += sph_factor * dt * F_b; the attached particle takes the boid's
                                velocity every step (it is kinematic) */
#define SPH_COUPLE_LITERAL 1 /* the paper's velocity update read literally: the attached particle keeps
                                its own velocity and is integrated like every particle (its fluid
                                force F_b plus gravity), only its position follows the boid, and
                                v_b += sph_factor * v_att (section "Boid Motion and Agent Fluid
                                Interaction"); sph_set_state resets v_att to the boid's velocity */

/* Bits of the sticky device error word (sph_status). */
#define SPH_DEV_NONFINITE 1u  /* a density, position or velocity became NaN/Inf  */
#define SPH_DEV_CLAMPED   2u  /* a fluid position lay outside the tank (or was NaN) when binned; its cell was clamped */
#define SPH_DEV_TIMEOUT   4u  /* a bounded wait inside a kernel gave up          */
#define SPH_DEV_LIST_OVERFLOW 8u /* a neighbour list did not fit the pair buffer  */
#define SPH_DEV_BOUNDS   16u  /* bounds-checked builds only: a sorted-slot index of a walk or of
                                 a hit segment was out of range; the access was skipped   */

/* Fields that sph_get_fields can return (one per call). */
#define SPH_FIELD_RHO         0  /* float[n_tot]   density, by particle id                 */
#define SPH_FIELD_PRESSURE    1  /* float[n_tot]   k (rho - rho0), by particle id          */
#define SPH_FIELD_ACC         2  /* float4[n_tot]  acceleration, by particle id            */
#define SPH_FIELD_TOUCHED     3  /* int[n_tot]     touched_by_boid, by particle id          */
#define SPH_FIELD_INFLUENCE   4  /* float4[n_tot]  boid_influence, by particle id           */
#define SPH_FIELD_NBR_COUNT   5  /* int[n_tot]     neighbour count (self excluded), by id   */
#define SPH_FIELD_KEYS        6  /* uint[n_tot]    cell key of the step's binning, by id    */
#define SPH_FIELD_PERM        7  /* int[n_tot]     id at each sorted slot                   */
#define SPH_FIELD_CELL_START  8  /* uint[ncells+1] first sorted slot of each cell           */
#define SPH_FIELD_FB          9  /* float4[n_boid] fluid force F_b on each boid             */
#define SPH_FIELD_BOID_KEYS  10  /* uint[n_boid]   boid-grid cell key, by boid id           */
#define SPH_FIELD_BOID_PERM  11  /* int[n_boid]    boid id at each sorted boid slot         */
#define SPH_FIELD_BOID_CELL_START 12 /* uint[nbcells+1] first sorted boid slot per cell    */
#define SPH_FIELD_NCAND      13  /* int[n_tot]     candidates the density pass tested, by id */
#define SPH_FIELD_FALLBACK   14  /* int[n_boid]    1 where the last surrogate call used the exact path */
#define SPH_FIELD_OBSTACLE_GRID 15 /* float4[nbcells] mean obstacle normal (xyz) and count (w) per boid-grid cell */
#define SPH_FIELD_NSEG       17  /* int[n_tot]     hit segments the density pass stored for the force pass,
                                    by id (0 for attached particles; above 128: the particle's candidates
                                    are tested again in the force pass) */
#define SPH_FIELD_ATT_VEL    16  /* float4[n_boid] velocity the attached particle of each boid carries into the
                                    next step (the boid's with SPH_COUPLE_FORCE, its own with SPH_COUPLE_LITERAL) */

/*
 * Parameters of a scene.  Paper notation: h smoothing length, rho0 rest
 * density, k gas constant (p = k (rho - rho0)), mu viscosity, mass particle
 * mass (every particle, attached ones included), d = cell_size the grid
 * cell (d >= h/4; the walk visits every cell the h-sphere can reach, 27 of
 * them for d >= h, clipped per particle for smaller cells), boid radii
 * r_sep ("protect_range") and r_vis ("visible_range"), rule weights w_sep
 * ("sep"), w_align ("mat"), w_coh ("cen"), sph_factor, the speed limits
 * v_min / v_max, edge_turn (edge avoidance), boid_cell_size (>= r_vis/4).
 * The paper gives no value for the boid weights, the wall restitution or
 * the edge turn; they are free parameters.
 */
typedef struct sph_params {
    float h, rho0, k, mu, dt, gx, gy, gz, mass;
    float box_min[3], box_max[3];
    float cell_size;
    int   const_set;           /* SPH_MULLER3D | SPH_PAPER_LITERAL */
    float wall_restitution;    /* walls: x reflected, v_n <- -wall_restitution v_n */
    float r_sep, r_vis, w_sep, w_align, w_coh, sph_factor, v_min, v_max, edge_turn;
    float boid_cell_size;
    int   coupling_mode;       /* SPH_COUPLE_FORCE (default) or SPH_COUPLE_LITERAL */
    float cell_size_x;         /* particle-grid cell size along x; 0: cell_size (cubic cells) */
} sph_params;

typedef struct sph_handle sph_handle;

/*
 * Bytes of device workspace a scene of n_fluid + n_boid particles needs
 * (all per-step arrays, the double-buffered SoA state and the grids).
 * Errors: SPH_ERR_ARG for invalid parameters (see sph_create), a NULL
 * `bytes` or negative counts; SPH_ERR_OVERFLOW if the grid or the counts
 * exceed 2^31 - 1.
 */
int sph_workspace_size(const sph_params* p, int n_fluid, int n_boid, size_t* bytes);

/*
 * Grid dimensions dim = ceil((box_max - box_min) / cell), per axis, of the
 * particle grid (which = 0, cell = cell_size) or the boid grid (which = 1,
 * cell = boid_cell_size) (section "Neighborhood Search").
 */
int sph_grid_dims(const sph_params* p, int which, int dims[3]);

/*
 * Particle mass that makes the density of an infinite cubic lattice of the
 * given spacing equal rho0 under the poly6 kernel (self term included):
 * mass = rho0 / sum_o W_poly6(|o| spacing), o over integer offsets with
 * |o| spacing < h.  Host-side computation in double; no device work.
 */
int sph_lattice_mass(const sph_params* p, float spacing, float* mass);

/*
 * Create a scene handle on a caller-owned device workspace of ws_bytes
 * (>= sph_workspace_size, 256-byte aligned).  The current CUDA device must
 * be the workspace's device.  The state is undefined until sph_set_state.
 * Errors: SPH_ERR_ARG if h, rho0, mass, dt <= 0, cell_size < h/4,
 * boid_cell_size < r_vis/4, r_sep > r_vis, box_max <= box_min on an axis,
 * an unknown const_set / coupling_mode, a small or misaligned workspace.
 */
int sph_create(const sph_params* p, int n_fluid, int n_boid, void* workspace,
               size_t ws_bytes, sph_handle** out);

/*
 * Batched scenes: S independent scenes (own parameters, own counts) in one
 * handle.  Every pass of sph_step then runs as one launch over the particles
 * (or boids, or cells) of all scenes, and each scene's result is bitwise the
 * result of that scene run alone.  The state arrays of sph_set_state /
 * sph_get_state are the scenes' arrays concatenated in scene order (fluid:
 * scene 0's n_fluid[0] particles, then scene 1's ...; boids likewise).
 * Particle ids of the fields are global: the attached particle of boid b
 * (b counted over the concatenated boids) has id b, fluid particle f (over the
 * concatenated fluid) has id n_boid_total + f; cell keys are global (scene
 * k's cells follow scene k-1's).  For S = 1 this is exactly sph_create.
 * Errors: as sph_create for any scene, SPH_ERR_ARG for S < 1 or NULL arrays,
 * SPH_ERR_OVERFLOW beyond 2^31 - 1 particles or cells in total.
 */
int sph_batch_workspace_size(const sph_params* params, const int* n_fluid, const int* n_boid, int S,
                             size_t* bytes);
int sph_batch_create(const sph_params* params, const int* n_fluid, const int* n_boid, int S,
                     void* workspace, size_t ws_bytes, sph_handle** out);

/*
 * Launch shape of the two neighbour passes (section "Neighbor Search with
 * Sorting": the density pass and the force pass each search the sorted
 * grid): `block` threads per block (64, 128, 256 or 512), and where the
 * force pass takes its pairs from.  use_segments = 1 (the default): the
 * density pass, which tests every candidate anyway, records each fluid
 * particle's force pairs as segments (first sorted slot, 32-bit mask) in
 * walk order, and the force pass reads them instead of testing the
 * candidates again (1 KiB of workspace per particle holds them; a
 * particle with more than 128 segments is tested again).  use_segments = 0:
 * the force pass tests the candidates itself.  Neither choice changes any
 * result bit: the pairs and their order are the same.  Errors: SPH_ERR_ARG.
 */
int sph_set_tuning(sph_handle* h, int block, int use_segments);

/*
 * Particles per thread of the two neighbour passes' separate launches (the
 * trade-off of section "Experimental Results": fewer threads, each taking
 * several particles): ppt = 1 (the default), 2 or 4; thread t of a grid of
 * T threads takes particles t, t + T, ...  No result bit changes.  The fused
 * pipeline (sph_set_pipeline) takes its own tiles.  Errors: SPH_ERR_ARG.
 */
int sph_set_particles_per_thread(sph_handle* h, int ppt);

/*
 * Record the diagnostic fields in later steps: with record = 1 the force
 * pass also stores each particle's acceleration, touched_by_boid and
 * boid_influence (listing "Compute acceleration", section "Boid Motion and
 * Agent Fluid Interaction") for sph_get_fields; with record = 0 (the
 * default) it does not write them (36 bytes per particle and step less),
 * and SPH_FIELD_ACC, SPH_FIELD_TOUCHED and SPH_FIELD_INFLUENCE fail with
 * SPH_ERR_STATE until a step is taken with record = 1.  The step's results
 * (state, densities, F_b) are the same either way.  A captured step
 * (sph_graph_step) is captured again after a change.  Errors: SPH_ERR_ARG.
 */
int sph_set_diagnostics(sph_handle* h, int record);

/*
 * Both neighbour passes in one persistent launch (the batched step's
 * pass over (scene, tile) work items; section "Experimental Results" tunes
 * the threads per group of the paper's dispatches).  tile_slots > 0: one
 * cooperative launch whose resident CTAs take tiles of tile_slots
 * consecutive sorted slots (runs of cells, across the scenes) from an
 * atomic queue for the density pass, meet at a grid barrier, then take the
 * boids (a warp each: F_b) and the tiles again for the force pass; block:
 * threads per CTA (128 or 256).  The barrier's wait is bounded (about 2^31
 * SM clock cycles, a second): a CTA that gives up sets SPH_DEV_TIMEOUT and
 * returns, leaving the step unfinished but the device usable.  Results are
 * bit for bit those of the separate launches.  tile_slots = 0 (the
 * default): separate launches.  The neighbour lists (sph_set_neighbor_lists)
 * take the separate launches.  A captured step is captured again.
 * Errors: SPH_ERR_ARG (tile_slots not 0 or a multiple of 32 in [32, 65536],
 * block not 128 or 256).
 */
int sph_set_pipeline(sph_handle* h, int tile_slots, int block);

/*
 * Test hook of the pipeline's bounded wait: with cta >= 0 that CTA of later
 * fused launches does not arrive at the grid barrier, so every CTA gives up
 * at its limit and the step ends with SPH_DEV_TIMEOUT set (no fault, the
 * context stays usable; the step's state is then unspecified: load a state
 * again).  cta = -1 (the default) turns it off.  Errors: SPH_ERR_ARG.
 */
int sph_debug_barrier_skip(sph_handle* h, int cta);

/*
 * Load the state: fluid_pos4 / fluid_vel4 hold n_fluid float4 (fluid order),
 * boid_pos4 / boid_vel4 hold n_boid float4 (boid order).  on_host = 1: host
 * buffers (copied on `stream`, which is synchronised before returning);
 * on_host = 0: device buffers, 16-byte aligned.  Any pointer of an empty
 * set may be NULL.  Errors: SPH_ERR_ARG (NULL or misaligned pointer),
 * SPH_ERR_CUDA.
 */
int sph_set_state(sph_handle* h, const float* fluid_pos4, const float* fluid_vel4,
                  const float* boid_pos4, const float* boid_vel4, int on_host, void* stream);

/* Store the current state into the same layouts as sph_set_state. */
int sph_get_state(sph_handle* h, float* fluid_pos4, float* fluid_vel4,
                  float* boid_pos4, float* boid_vel4, int on_host, void* stream);

/*
 * Advance nsteps whole steps on `stream` (asynchronous; no host sync, no
 * allocation).  One step: attach particles to boids; bin (keys, counting
 * sort by cell then particle id); density + pressure; pair forces,
 * touched_by_boid, boid_influence and the fluid force F_b on each boid;
 * boid rules (start-of-step snapshot, rules in the listed order, then
 * v_b += sph_factor dt F_b, edge avoidance, speed limit, x_b += v_b dt);
 * Euler-Cromer integration of the fluid with damped wall reflection.
 * With boids (and without the fused pipeline of sph_set_pipeline), the
 * boids' binning, F_b and rules run on a stream the handle owns, forked from
 * `stream` at the start of each step and joined back into it before the
 * step ends: to the caller the work is ordered on `stream` as if it ran
 * there alone (a capture of `stream` takes the side branch with it), and the
 * results are bit for bit those of the serial order.
 * Errors: SPH_ERR_ARG (nsteps < 0), SPH_ERR_STATE (no state loaded),
 * SPH_ERR_CUDA.  Device-side anomalies set bits of the error word.
 */
int sph_step(sph_handle* h, int nsteps, void* stream);

/*
 * sph_step through a CUDA graph: the first call captures one step on
 * `stream` (which must not be the legacy default stream) and later calls
 * replay it, nsteps times, with the same results as sph_step.  A change of
 * stream or tuning recaptures.  Per-pass event timing is not recorded in
 * graph mode.  Errors: SPH_ERR_ARG, SPH_ERR_STATE, SPH_ERR_CUDA.
 */
int sph_graph_step(sph_handle* h, int nsteps, void* stream);

/*
 * Fluid force on every boid for the CURRENT state, written as n_boid float4
 * to out_f4 (device, 16-byte aligned); the state is not changed.  Modes:
 *   SPH_BOID_EXACT: F_b = (1/rho_b) sum_j f_bj over the fluid neighbours j of
 *     the boid's attached particle (section "Boid Motion and Agent Fluid
 *     Interaction"), from a density pass over every particle; w = 0.
 *   SPH_BOID_EXACT_LOCAL: the same forces, bit for bit, computing densities
 *     only for the attached particles and their fluid neighbours; w = 0.
 *   SPH_BOID_SURROGATE: the attached surrogate network (sph_set_surrogate)
 *     on the boids' stencil features (sph_features): F_b = y[0:3] * f_scale,
 *     w = 0.
 *   SPH_BOID_SURROGATE_FALLBACK: the surrogate, except for the boids whose
 *     error head y[3] exceeds log_err_max (or whose output is not finite):
 *     those get the exact-local force and w = 1.
 * Errors: SPH_ERR_ARG (mode, out), SPH_ERR_STATE (no state, or no surrogate
 * for the surrogate modes), SPH_ERR_CUDA.
 */
#define SPH_BOID_EXACT              0
#define SPH_BOID_SURROGATE          1
#define SPH_BOID_SURROGATE_FALLBACK 2
#define SPH_BOID_EXACT_LOCAL        3
int sph_boid_forces(sph_handle* h, int mode, float* out_f4, void* stream);

/*
 * sph_boid_forces through a CUDA graph, one per mode: the first call of a
 * mode runs plainly (it also does the mode's one-time set-up), the next
 * captures the call's launches on `stream` (not the legacy default stream)
 * and every later call replays them: the same forces, bit for bit, for a
 * fraction of the launch overhead.  A change of stream or out pointer
 * recaptures; so does sph_set_surrogate, sph_set_surrogate_bounds or
 * sph_set_tuning.  A state whose cell keys are not yet computed (just
 * loaded) takes the plain path.  Errors: as sph_boid_forces, and
 * SPH_ERR_ARG for the default stream.
 */
int sph_graph_boid_forces(sph_handle* h, int mode, float* out_f4, void* stream);

/*
 * Stencil features of every boid for the CURRENT state (the surrogate's
 * input): x_out holds n_boid rows of SPH_MLP_IN BF16 (device, 16-byte
 * aligned).  Row b: the 4 x 4 x 4 cells of size h of a grid anchored at
 * box_min, from c0 = floor((p_b - box_min) / h - 1.5) per axis; cell
 * q = (iz * 4 + iy) * 4 + ix gives columns 4q .. 4q+3 = (fluid particles in
 * the cell * mass / (h^3 rho0), their mean velocity); columns 256 .. 258:
 * the boid's velocity; 259 .. 261: its offset from the stencil's centre,
 * (p_b - box_min) / h - c0 - 2; 262: the density of its attached particle
 * / rho0; 263: S0 = m / (rho0 h^3) sum (1 - q); 264 .. 266: S1 = m / (rho0
 * h^3) sum (1 - q) (v_j - v_b); 267 .. 269: S2 = m / (rho0 h^3) sum
 * (1 - q)^2 (p_b - x_j) / r, over the fluid particles j within h
 * (q = r / h); 270, 271: zero.  Errors: SPH_ERR_ARG, SPH_ERR_STATE,
 * SPH_ERR_CUDA.
 */
int sph_features(sph_handle* h, void* x_out, void* stream);

/*
 * Attach a surrogate network (NULL detaches) for the surrogate modes of
 * sph_boid_forces: forces are the network's outputs 0..2 times f_scale;
 * boids whose error-head output exceeds log_err_max take the exact path in
 * SPH_BOID_SURROGATE_FALLBACK.  The network must stay alive while attached.
 */
typedef struct sph_mlp sph_mlp;
int sph_set_surrogate(sph_handle* h, sph_mlp* m, float f_scale, float log_err_max);
/*
 * Input range of the surrogate (the gate's out-of-range check): with lo and
 * hi set (device, SPH_MLP_IN floats each, the caller's; NULL turns the
 * check off), a boid any of whose features lies outside [lo, hi] is flagged
 * for the exact path like one whose error head is too high.  Errors:
 * SPH_ERR_ARG (only one of lo, hi given).
 */
int sph_set_surrogate_bounds(sph_handle* h, const float* lo, const float* hi);

/*
 * Copy one field of the most recent step (SPH_FIELD_*) to `out` (device,
 * or host with on_host = 1), sized as listed with the SPH_FIELD_* codes.
 * Errors: SPH_ERR_ARG (unknown field, NULL out), SPH_ERR_STATE (no step
 * since the last sph_set_state; or acc, touched, influence requested after a
 * step taken without sph_set_diagnostics(h, 1)), SPH_ERR_CUDA.
 */
int sph_get_fields(sph_handle* h, int field, void* out, int on_host, void* stream);

/*
 * The fixed-capacity hash grid of section "Neighborhood Search", as an
 * ablation of the exact search: every particle appends its index to its
 * cell's bucket through an atomic counter, a bucket keeps at most
 * `capacity` indices and drops the rest, and each particle counts its
 * neighbours (the exclusions of sph_debug_neighbors) over the cells within
 * ceil(h / cell_size) of its own.  counts: device int per particle id
 * (n_fluid + n_boid); *dropped (device, 8-byte aligned): the particles the
 * buckets lost; scratch: device, 4-byte aligned, at least
 * ncells * (1 + capacity) * 4 bytes.  Equal to sph_debug_neighbors' counts
 * when no cell holds more than `capacity` particles; test hook, not part of
 * the step.  Errors: SPH_ERR_ARG, SPH_ERR_STATE, SPH_ERR_CUDA.
 */
int sph_debug_bucket_neighbors(sph_handle* h, void* scratch, size_t bytes, int capacity, int* counts,
                               unsigned long long* dropped, void* stream);

/*
 * Test hook: bin the CURRENT state and write every particle's neighbour
 * list, N(i) = { j != i : not both attached, r_ij^2 < h^2 } with the float32
 * predicate, in the order the 27-cell walk visits them (cells dz, dy, dx
 * ascending; particles of a cell by id).  counts: int[n_tot] by id (device).
 * If offsets (int64[n_tot + 1], device, by id) and list (int[offsets[n_tot]],
 * device) are non-NULL, list[offsets[i] ..] receives the ids.  State is
 * unchanged.  Errors: SPH_ERR_ARG, SPH_ERR_STATE, SPH_ERR_CUDA.
 */
int sph_debug_neighbors(sph_handle* h, int* counts, const long long* offsets, int* list,
                        void* stream);

/*
 * Per-step diagnostics (the step's optional statistics row): for every scene
 * k, from the state after the most recent step and that step's fields,
 * out[k * SPH_STATS_N + i] (float64; device, or host with on_host = 1, which
 * synchronises the stream) with i =
 *   SPH_STAT_FLUID      fluid particles of the scene
 *   SPH_STAT_NBR_MEAN   mean neighbour count of its fluid particles (self
 *                       excluded; section "Neighborhood Search")
 *   SPH_STAT_NBR_MAX    largest neighbour count of a fluid particle
 *   SPH_STAT_CELL_MAX   most particles (attached included) in one cell of
 *                       the step's binning
 *   SPH_STAT_MOM_X..Z   sum of m v over its fluid particles after the step
 *   SPH_STAT_KE         kinetic energy (1/2) m sum |v|^2 of the fluid after
 *                       the step
 *   SPH_STAT_RHO_MIN, SPH_STAT_RHO_MAX, SPH_STAT_RHO_MEAN
 *                       the fluid particles' densities of the step
 *   SPH_STAT_SPEED_MAX  largest fluid speed after the step
 * (means, density bounds: 0 for a scene without fluid).  Counts and the
 * neighbour sum are integers, extrema exact; the other sums are float64 over
 * float32 partial sums of at most 8 values, all in a fixed order: the same
 * state gives the same bits, whatever else is in the batch.  Two kernel launches; no allocation, graph-capturable with
 * on_host = 0.  Errors: SPH_ERR_ARG (NULL), SPH_ERR_STATE (no step since
 * the state was loaded), SPH_ERR_CUDA.
 */
#define SPH_STATS_N        12
#define SPH_STAT_FLUID      0
#define SPH_STAT_NBR_MEAN   1
#define SPH_STAT_NBR_MAX    2
#define SPH_STAT_CELL_MAX   3
#define SPH_STAT_MOM_X      4
#define SPH_STAT_MOM_Y      5
#define SPH_STAT_MOM_Z      6
#define SPH_STAT_KE         7
#define SPH_STAT_RHO_MIN    8
#define SPH_STAT_RHO_MAX    9
#define SPH_STAT_RHO_MEAN  10
#define SPH_STAT_SPEED_MAX 11
int sph_stats(sph_handle* h, double* out, int on_host, void* stream);

/*
 * Read (and keep) the sticky device error word into *bits; synchronises the
 * handle's last stream.  sph_clear_status zeroes it (asynchronously).
 */
int sph_status(sph_handle* h, unsigned* bits);
int sph_clear_status(sph_handle* h, void* stream);

/* Message of the last failure on h (or of handle-less calls if h is NULL). */
const char* sph_last_error(sph_handle* h);

/* Number of kernels this handle has launched since creation. */
long long sph_launch_count(sph_handle* h);

/*
 * Per-pass CUDA-event timing of sph_step (the library's tracing hook).
 * Kinds: SPH_KIND_KEYS (cell keys of a freshly loaded state), SPH_KIND_SCAN
 * (exclusive scan of the cell counts), SPH_KIND_SCATTER, SPH_KIND_SORT
 * (per-cell sort + gather), SPH_KIND_DENSITY, SPH_KIND_FORCES (pair forces
 * + integration + next keys), SPH_KIND_BOID_BIN (boid-grid binning),
 * SPH_KIND_BOID_RULES, SPH_KIND_LISTS, SPH_KIND_FEATURES, SPH_KIND_PIPELINE
 * (SPH_NUM_KINDS kinds).  sph_profile_enable(h, n) creates a host-side pool
 * of 2n events (n = 0 disables and frees it); while enabled, each pass of
 * sph_step is bracketed by two events recorded on the step's stream, up to
 * n passes.  sph_profile_read synchronises on the last event and writes,
 * per kind (nkinds entries), the summed milliseconds and the number of
 * passes, then restarts the record.  Errors: SPH_ERR_ARG, SPH_ERR_CUDA.
 */
#define SPH_KIND_KEYS       0
#define SPH_KIND_SCAN       1
#define SPH_KIND_SCATTER    2
#define SPH_KIND_SORT       3
#define SPH_KIND_DENSITY    4
#define SPH_KIND_FORCES     5
#define SPH_KIND_BOID_BIN   6
#define SPH_KIND_BOID_RULES 7
#define SPH_KIND_LISTS      8  /* neighbour lists: offsets scan + fill (when set) */
#define SPH_KIND_FEATURES   9  /* the surrogate's stencil features (sph_features, surrogate modes) */
#define SPH_KIND_PIPELINE  10  /* both neighbour passes in one launch (sph_set_pipeline) */
#define SPH_NUM_KINDS      11
int sph_profile_enable(sph_handle* h, int max_passes);
int sph_profile_read(sph_handle* h, double* ms, long long* passes, int nkinds);

/*
 * Neighbour lists, an alternative to testing candidates in the force pass
 * (the list-building neighbour search of section "Neighborhood Search";
 * an ablation of the walk).  With a pair buffer set, every sph_step scans
 * the density pass's neighbour counts into per-particle offsets, writes
 * each particle's neighbours (fluid particles: every particle within h but
 * itself; attached particles: the fluid ones), in walk order, into the
 * buffer, and the force pass reads a fluid particle's list instead of
 * testing its candidates: results are bit-identical to the walk.
 * pair_buffer: device memory, 4-byte aligned, bytes / 4 entries (one per
 * ordered neighbour pair, i.e. the sum of the neighbour counts is needed).
 * A particle whose list would end beyond the buffer tests its candidates as
 * without lists and sets SPH_DEV_LIST_OVERFLOW.  NULL (or bytes < 4) turns
 * the lists off (the default).  The buffer stays the caller's and must
 * outlive its use.  Errors: SPH_ERR_ARG.
 */
int sph_set_neighbor_lists(sph_handle* h, void* pair_buffer, size_t bytes);

/* Free the host-side handle (the workspace stays the caller's). */
void sph_destroy(sph_handle* h);

/*
 * Boid-force surrogate (not in the paper): an MLP from a boid's local flow
 * features to the fluid force F_b of the SPH coupling.  Rows of x are
 * SPH_MLP_IN BF16 features (256 stencil features, 3 boid-velocity features,
 * zero padding); y rows are SPH_MLP_OUT FP32 outputs (0..2: F_b / F_scale,
 * 3: error head, log10 of the expected relative error; the rest unused).
 * Layers 272 -> 256 -> 256 -> 256 -> 16 with exact-erf GELU between them.
 * Parameters are one FP32 vector of SPH_MLP_PARAMS floats in the order
 * W1 [256][272], b1, W2 [256][256], b2, W3, b3, W4 [16][256], b4.  Every
 * matrix product runs on the tensor cores (BF16 operands, FP32 accumulate);
 * training is Adam on FP32 master weights.  A handle owns a caller-given
 * workspace sized for batches of up to max_batch rows (a multiple of 128);
 * every batch B must be a positive multiple of 128 and <= max_batch.
 */
#define SPH_MLP_IN      272
#define SPH_MLP_HIDDEN  256
#define SPH_MLP_OUT     16
#define SPH_MLP_PARAMS  205584
int sph_mlp_workspace_size(int max_batch, size_t* bytes);
int sph_mlp_create(int max_batch, void* workspace, size_t ws_bytes, sph_mlp** out);
void sph_mlp_destroy(sph_mlp* m);
/* Load parameters (device FP32 vector) and reset the Adam moments. */
int sph_mlp_set_params(sph_mlp* m, const float* params, void* stream);
int sph_mlp_get_params(sph_mlp* m, float* params, void* stream);
/*
 * The optimiser's state after the last sph_mlp_train_step (or
 * sph_mlp_gradients): grads, the gradient of the last step, and m1, m2, the
 * first and second Adam moments (Kingma and Ba; beta1 = 0.9, beta2 = 0.999,
 * eps = 1e-8 as float32, bias corrections 1 - beta^t rounded once from
 * double), packed like the parameters (SPH_MLP_PARAMS FP32 each, device,
 * copied on `stream`); *step (host): the Adam steps taken since the last
 * sph_mlp_set_params.  For checkpoints and for checking the update against
 * a reference.  Errors: SPH_ERR_ARG (NULL pointer), SPH_ERR_CUDA.
 */
int sph_mlp_get_optimizer_state(sph_mlp* m, float* grads, float* m1, float* m2, long long* step, void* stream);
/*
 * Restore the Adam moments and step count of a checkpoint (after
 * sph_mlp_set_params, which resets them): with the parameters, m1, m2 and
 * step as sph_mlp_get_optimizer_state gave them, the next train steps are
 * bit for bit those the saved network would have taken.  Device FP32
 * vectors of SPH_MLP_PARAMS, copied on `stream`.  Errors: SPH_ERR_ARG (NULL
 * pointer, step < 0), SPH_ERR_CUDA.
 */
int sph_mlp_set_optimizer_state(sph_mlp* m, const float* m1, const float* m2, long long step, void* stream);
/* y[B][16] = MLP(x[B][272]) (device buffers; x 16-byte aligned). */
int sph_mlp_forward(sph_mlp* m, const void* x_bf16, int B, float* y, void* stream);
/* Parameter gradients of sum(dy * y) for an upstream gradient dy[B][16]
 * (FP32, device), written to grads (SPH_MLP_PARAMS FP32, device). */
int sph_mlp_gradients(sph_mlp* m, const void* x_bf16, const float* dy, int B, float* grads, void* stream);
/* One Adam step on a batch: targets t[B][4] (0..2 force / F_scale, 3 error
 * target).  phase 0: force loss mean 1/2 |y[0:3] - t[0:3]|^2, every
 * parameter except the error head (row 3 of W4, b4[3]); phase 1: error loss
 * mean 1/2 (y[3] - t[3])^2, the error head only.  *loss_out (device, may be
 * NULL) receives the batch loss. */
int sph_mlp_train_step(sph_mlp* m, const void* x_bf16, const float* target, int B, int phase, float lr,
                       float* loss_out, void* stream);
/* Sticky device error word of the MLP kernels (SPH_DEV_TIMEOUT); syncs. */
int sph_mlp_status(sph_mlp* m, unsigned* bits, void* stream);
long long sph_mlp_launch_count(sph_mlp* m);
/*
 * Test hook of the activation the network's kernels use: out[i] = GELU(z[i])
 * (grad = 0) or GELU'(z[i]) (grad = 1) for n floats in device memory, GELU
 * the exact-erf form (z Phi(z)), erf evaluated by formula 7.1.26 of
 * Abramowitz and Stegun (absolute error <= 1.5e-7 plus float32 rounding);
 * grad = 2: GELU(z[i]) by the packed two-value form of the same formula that
 * the fused inference kernel uses.
 * Errors: SPH_ERR_ARG (NULL pointers, n < 0, grad not 0/1/2), SPH_ERR_CUDA.
 */
int sph_debug_gelu(const float* z, int n, int grad, float* out, void* stream);
/*
 * Test hook of the tensor-core GEMM: for BF16 row-major A[M][K] (leading
 * dimension lda) and B[N][K] (ldb), both 16-byte aligned with leading
 * dimensions multiples of 8, N a multiple of 4 and C 16-byte aligned
 * (SPH_ERR_ARG otherwise), writes the FP32 partial products of `splits`
 * K-ranges to C[split][M][N] (C holds splits * M * N floats; their sum is
 * A B^T; the actual number of splits is min(splits, ceil(K / 64)) rounded
 * so that no range is empty).  err: a device word for SPH_DEV_TIMEOUT.
 */
int sph_debug_gemm(const void* A, int lda, const void* B, int ldb, int M, int N, int K, int splits, float* C,
                   unsigned* err, void* stream);

/* ---------------------------------------------------------- obstacles
 * Obstacle avoidance of the boids (section "Boid Motion and Agent Fluid
 * Interaction": an obstacle grid holds the normals of the obstacles'
 * meshes; a boid steers by the averaged normals of the obstacle cells
 * within its visual range, those within its protection range weighted
 * more).  Analytic obstacles stand in for the meshes: spheres (host array
 * of n_sphere x (centre x, y, z, radius > 0)) and boxes (host array of
 * n_box x (min x, y, z, max x, y, z)), at most SPH_MAX_OBSTACLES together.
 * The obstacle grid has the boid grid's cells; an obstacle counts in a cell
 * when its signed distance at the cell's centre fl(min + fl((i + 0.5) d))
 * is within half a cell diagonal (fl(0.8660254 d)), and adds its outward
 * unit normal at the surface point nearest the centre (inside a box: the
 * normal of its nearest face); each cell keeps the mean and the count
 * (SPH_FIELD_OBSTACLE_GRID).  Each step, after the fluid coupling and before
 * the edge avoidance and the speed limit, a boid adds
 * w_obst * (sum over the obstacle cells whose centre is within r_vis of
 * it of w_c * mean normal_c) / (their number), w_c = near_factor within
 * r_sep and 1 beyond (the float32 distance predicate of the boid pairs).
 * n_sphere = n_box = 0 turns the term off.  Single-scene handles only; the
 * call waits for its own copies on `stream`, so make it outside any stream
 * capture.  Errors: SPH_ERR_ARG (bad counts, NULL arrays, a radius <= 0, a
 * box with max < min, non-finite values, near_factor < 0, a batched
 * handle), SPH_ERR_CUDA.
 */
#define SPH_MAX_OBSTACLES 256
int sph_set_obstacles(sph_handle* h, const float* spheres, int n_sphere, const float* boxes, int n_box,
                      float w_obst, float near_factor, void* stream);

/* ------------------------------------------------------------ surface
 * Surface reconstruction from the particles (NEXT row of the scope: the
 * paper's third stage), headless: the triangles go to a device buffer.
 *
 * Voxel density (section "Voxel Density"): at every corner x of a grid,
 * phi(x) = |x - xbar| - r with xbar = sum_i w_i x_i,
 * w_i = k(|x - x_i| / R) / sum_j k(|x - x_j| / R), k(s) = (1 - s^2)^3, over
 * the fluid particles with |x - x_i| < R (decided in float32 like the step's
 * neighbour predicate, R for h; boid-attached particles are not fluid); r is
 * the particle radius; a corner without neighbours gets phi = R.  Corner
 * (ix, iy, iz) lies at fl(origin + fl(i * spacing)) per axis and is element
 * ix + nx (iy + ny iz).
 *
 * sph_voxel_grid: the corner grid covering p's box with ceil(R / spacing) + 1
 * corners beyond it on every side (those are farther than R from any
 * particle in the box, so the surface closes inside the grid): origin[3],
 * dims[3] (corners per axis).  Errors: SPH_ERR_ARG (spacing or radius not
 * > 0, empty box), SPH_ERR_OVERFLOW (more than 2^31 - 1 corners).
 *
 * sph_voxel_density: phi (device float array of nx ny nz) and, if counts
 * is not NULL, the neighbour count of every corner (device int array), for
 * the state the handle holds, enqueued on `stream`.  Single-scene handles
 * only.  Errors: SPH_ERR_ARG (NULL, misaligned (4 bytes) or bad sizes,
 * batched handle), SPH_ERR_OVERFLOW (> 2^31 - 1 corners), SPH_ERR_STATE (no
 * state), SPH_ERR_CUDA.  Like sph_features, it re-bins the state and
 * invalidates the step's fields.
 */
int sph_voxel_grid(const sph_params* p, float spacing, float radius, float origin[3], int dims[3]);
int sph_voxel_density(sph_handle* h, const float origin[3], const int dims[3], float spacing, float radius,
                      float particle_radius, float* phi, int* counts, void* stream);
/*
 * Marching cubes (section "Marching Cubes") over a corner grid of float32
 * values phi (device, nx ny nz, layout as above): cube (ix, iy, iz) has
 * vertex v at corner (ix, iy, iz) + (0,0,0), (1,0,0), (1,1,0), (0,1,0),
 * (0,0,1), (1,0,1), (1,1,1), (0,1,1) for v = 0..7 and edges (v0 v1),
 * (v1 v2), (v2 v3), (v3 v0), (v4 v5), (v5 v6), (v6 v7), (v7 v4), (v0 v4),
 * (v1 v5), (v2 v6), (v3 v7) (the numbering of the paper's worked example);
 * its cube index has bit v set when phi at vertex v is below iso; a cut
 * edge's vertex is p1 + (iso - v1) / (v2 - v1) (p2 - p1), p1 its endpoint of
 * smaller coordinate.  The triangles of the generated table (sph_mc_tables)
 * go to tris as 9 floats each (three vertices x, y, z), cubes in order of
 * their index ix + (nx-1) (iy + (ny-1) iz), each cube's triangles in table
 * order; triangles wind so that their right-hand normal points to the side
 * below iso.  At most max_tris are written; *ntri (a device unsigned)
 * receives the total, which may exceed max_tris (saturated at 0xfffffffe).
 * Three launches: the triangle counts of tiles of 1,024 cubes, one scan of
 * the tile totals, then each tile's triangles from its offset, spread
 * evenly over the tile's threads.  workspace: device memory of
 * sph_mc_workspace_size bytes, 256-byte aligned, owned by the caller.
 * The first call on a device copies the tables to its memory
 * (synchronously); make it before any stream capture.  Errors: SPH_ERR_ARG
 * (NULL, misaligned, too small a workspace, spacing not > 0, iso not
 * finite), SPH_ERR_OVERFLOW (more than 2^31 - 1 corners or (2^31 - 1) / 5
 * cubes), SPH_ERR_CUDA.  Messages in sph_last_error(NULL).
 */
int sph_mc_workspace_size(const int dims[3], size_t* bytes);
int sph_marching_cubes(const float* phi, const int dims[3], const float origin[3], float spacing, float iso,
                       void* workspace, size_t ws_bytes, float* tris, long long max_tris, unsigned* ntri,
                       void* stream);
/*
 * Host copies of the marching-cubes tables the library generates from the
 * cube's numbering: edge_table[256] (bit e set when edge e is cut) and
 * tri_table[256][16] (edge triples, -1 terminated; at most 5 triangles).
 * A face with four cut edges is split around each of its corners below the
 * isovalue (a rule of the face alone, so neighbouring cubes agree and the
 * surface closes).  Either pointer may be NULL.  Errors: SPH_ERR_CUDA if
 * the generator fails its own consistency checks.
 */
int sph_mc_tables(unsigned short* edge_table, signed char* tri_table);

/*
 * Allocation-free binning.  The paper has no counterpart to this entry point;
 * it exists for callers that cannot allocate device memory: code that runs
 * inside another framework's hook and owns only its input and output buffers
 * (the framework's allocator holds the rest of the device memory), or a
 * real-time loop where a cudaMalloc, which may synchronise the device, would
 * stall other streams.
 *
 * For n particles at pos4 (device float4, 16-byte aligned, by index; w
 * ignored) it bins them on the grid of sph_step (p->box_min/box_max/
 * cell_size, section "Neighbor Search with Sorting"): keys_out[n] the cell
 * key of each particle (by index), perm_out[n] the particle index at each
 * sorted slot (sorted by key, then index), cell_start_out[ncells + 1] the
 * first sorted slot of each cell (device arrays owned by the caller).
 * sph_step orders a cell by particle id instead of index; the two agree
 * where ids equal indices (a scene without boids whose state was just
 * loaded).  flags_out (device, 4-byte aligned; NULL: not reported) receives
 * this call's flag word: SPH_DEV_CLAMPED when a position lay outside the box
 * (or was NaN) and was binned into the nearest cell.  Work is enqueued on
 * `stream`.
 *
 * Its scratch is one file-scope device array of SPH_STATIC_SCRATCH_BYTES
 * (about 21 MiB) that every GPU which loads this library holds until the
 * process exits.  Limits: n <= SPH_STATIC_MAX_PARTICLES and a grid of at most
 * SPH_STATIC_MAX_CELLS cells; larger requests return SPH_ERR_ARG (message in
 * sph_last_error(NULL)) before any device work.  The array is shared by all
 * calls on a device and keeps the last call's contents; each call zeroes
 * what must start at zero.  Calls that overlap on the GPU race on it:
 * serialise them.  Every call looks up the array's address on the current
 * device (nothing is cached across calls, so a reset of the device's context
 * in between is harmless); the first call on a device may load the library's
 * device code there, so make it before any stream capture.  No device
 * memory is allocated or freed.
 */
#define SPH_STATIC_MAX_PARTICLES (1 << 22)
#define SPH_STATIC_MAX_CELLS     (1 << 20)
#define SPH_STATIC_SCRATCH_BYTES (21u << 20)
int sph_bin_static(const sph_params* p, int n, const float* pos4, unsigned* keys_out, int* perm_out,
                   unsigned* cell_start_out, unsigned* flags_out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SPH_GB300_H */
