/*
 * sph_oracle.c -- the CPU oracle of one SPH-with-boids step.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  The GPU library
 * never calls it and shares no code with it.
 *
 * What it is: a plain, slow restatement of the step in "A GPU-based
 * Hydrodynamic Simulator with Boid Interactions" (Liu, Kayar, Perlin,
 * arXiv 2311.15088), pass by pass, in the paper's order and notation:
 *
 *   1. attach one particle to every boid        (section "Boid Motion and Agent
 *                                                Fluid Interaction", particle
 *                                                attachment)
 *   2. bin particles into the uniform grid       (section "Neighborhood Search":
 *      with a counting sort                      get_cell, hash; section
 *                                                "Neighbor Search with Sorting":
 *                                                counts, prefix sum, scatter)
 *   3. density + equation of state               (section "Smoothed Particle
 *                                                Hydrodynamics": poly6 kernel;
 *                                                "Pressure and Viscosity": EOS)
 *   4. pressure + viscosity pair forces          ("Pressure and Viscosity":
 *      (+ touched_by_boid, boid_influence)       symmetrised pressure force,
 *                                                spiky gradient, viscosity
 *                                                Laplacian; listing "Compute
 *                                                acceleration")
 *   5. boid rules: separation, alignment,        ("Boid Motion and Agent Fluid
 *      cohesion, fluid coupling, edge            Interaction", items 1-6 and the
 *      avoidance, speed limit, position update   sph_factor coupling)
 *   6. Euler-Cromer integration + damped walls   (section "Governing
 *                                                Equations" frame loop; section
 *                                                "Background": damped boundary)
 *
 * Floating point: every value is computed in double from the float32 state.
 * Two things decide integers and are therefore evaluated exactly as the GPU
 * library evaluates them, in float32 with a fixed operation order:
 *   - the cell of a position: c = floor((p - min) * inv_d), inv_d = 1/d
 *     rounded to float once, clamped to [0, dim-1];
 *   - the neighbour predicate: dx = x_j - x_i per component (float), then
 *     r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx)) and r2 < h*h (h*h in float).
 * Build with -ffp-contract=off so that the compiler fuses nothing else.
 *
 * Readings of points the paper leaves open (documented in the design notes):
 *   - the 3-D normalised spiky / viscosity constants 45/(pi h^5) are the
 *     default; the printed 30/(pi h^4), 40/(pi h^4) (2-D normalisations) are
 *     const_set = 1;
 *   - a_i = (1/rho_i) * sum_j f_ij + g: the listing returns a force density;
 *   - density includes the self term m W(0); forces skip pairs with r2 == 0;
 *   - particles attached to boids see only fluid particles (no
 *     attached-attached pairs in density or force); they are kinematic;
 *   - the order inside a cell is the particle id (stable counting sort);
 *   - walls: reflect the position about the wall and scale the normal
 *     velocity by -wall_restitution, then clamp;
 *   - boids read a start-of-step snapshot; rules apply in the listed order;
 *   - obstacle avoidance (when obstacles are given): analytic spheres and
 *     boxes stand in for the obstacle meshes; their normals fill an obstacle
 *     grid over the boid grid's cells; a boid adds w_obst times the mean of
 *     the normals of the obstacle cells within its visual range (weighted
 *     near_factor within its protection range), after the fluid coupling
 *     and before the edge avoidance and the speed limit;
 *   - the voxel density and the corner grid of the surface stage: see
 *     or_voxel_density and oracle/surface.py.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846

typedef struct {
    double h, rho0, k, mu, dt, g[3], mass;
    double box_min[3], box_max[3], cell_size;
    int const_set;          /* 0: 3-D normalised constants, 1: printed (2-D) constants */
    double wall_restitution;
    double r_sep, r_vis, w_sep, w_align, w_coh, sph_factor, v_min, v_max, edge_turn;
    double boid_cell_size;
    int coupling_mode;      /* 0: force coupling; 1: the literal coupling (see or_step) */
    const void *obstacles;  /* const or_obstacles *, or NULL: no obstacle avoidance */
    const float *att_vel;   /* literal coupling: the attached particles' velocities (n_boid x 3)
                               going into the step; NULL: the boids' velocities */
    double cell_size_x;     /* particle-grid cell size along x; 0: cell_size */
} or_params;

/* Analytic obstacles standing in for the paper's obstacle meshes (section
 * "Boid Motion and Agent Fluid Interaction": the obstacle grid and obstacle
 * avoidance). */
typedef struct {
    int n_sphere, n_box;
    const float *sphere;    /* n_sphere x 4: centre x, y, z, radius */
    const float *box;       /* n_box x 6: min corner, max corner */
    double w_obst;          /* gain on the averaged normal */
    double near_factor;     /* weight of cells in the protection range */
} or_obstacles;

/* Outputs of or_step.  Any pointer may be NULL.  Particle ids: 0..n_boid-1
 * are the boid-attached particles, n_boid.. are fluid particles. */
typedef struct {
    double *rho, *pressure, *acc, *acc_scale, *influence;   /* per particle (acc, influence: 3) */
    int *touched, *nbr_count;                              /* per particle */
    unsigned *keys; int *perm; int *cell_start;            /* binning (cell_start: ncells+1) */
    double *new_fluid_pos, *new_fluid_vel;                 /* per fluid particle, 3 each */
    double *pre_wall_pos, *pre_wall_vel, *wall_margin;     /* per fluid particle */
    double *fb;                                            /* per boid, 3: fluid force on the boid */
    double *new_boid_pos, *new_boid_vel, *boid_vscale;     /* per boid */
    int *boid_nsep, *boid_nvis;                            /* per boid */
    unsigned *boid_keys; int *boid_perm; int *boid_cell_start;
    double *new_att_vel;                                   /* per boid, 3: the attached particle's
                                                              velocity going into the next step */
} or_outputs;

/* ------------------------------------------------------------------ grid */

typedef struct {
    int dim[3];
    long ncells;
    float minf[3];
    float inv_d, inv_dx;    /* 1/d along y and z, 1/dx along x */
} or_grid;

/* Number of cells per axis: dim = ceil((max - min) / d) (section
 * "Neighborhood Search"; the product dim_x dim_y dim_z is the cell count),
 * with cell size dx along x and d along y and z. */
static void grid_make_x(or_grid *g, const double mn[3], const double mx[3], double dx, double d)
{
    for (int a = 0; a < 3; ++a) {
        int n = (int)ceil((mx[a] - mn[a]) / (a == 0 ? dx : d));
        g->dim[a] = n < 1 ? 1 : n;
        g->minf[a] = (float)mn[a];
    }
    g->ncells = (long)g->dim[0] * g->dim[1] * g->dim[2];
    g->inv_d = 1.0f / (float)d;
    g->inv_dx = 1.0f / (float)dx;
}

static void grid_make(or_grid *g, const double mn[3], const double mx[3], double d)
{
    grid_make_x(g, mn, mx, d, d);
}

/* The particle grid's cell size along x. */
static double cell_x(const or_params *p) { return p->cell_size_x > 0.0 ? p->cell_size_x : p->cell_size; }

/* get_cell along one axis: floor((p - m) / d), in float32, clamped. */
static int cell_coord(const or_grid *g, int a, float x)
{
    float t = (x - g->minf[a]) * (a == 0 ? g->inv_dx : g->inv_d);
    float c = floorf(t);
    if (!(c >= 0.0f)) return 0;
    if (c >= (float)(g->dim[a] - 1)) return g->dim[a] - 1;
    return (int)c;
}

/* hash(c) = c_x + dim_x (c_y + dim_y c_z) (section "Neighborhood Search"). */
static long cell_hash(const or_grid *g, int cx, int cy, int cz)
{
    return (long)cx + (long)g->dim[0] * ((long)cy + (long)g->dim[1] * (long)cz);
}

static long key_of(const or_grid *g, const float *x)
{
    return cell_hash(g, cell_coord(g, 0, x[0]), cell_coord(g, 1, x[1]), cell_coord(g, 2, x[2]));
}

/* Counting sort (section "Neighbor Search with Sorting"): count particles per
 * cell, exclusive prefix sum -> cell offsets, then place particles.  Placing
 * them in increasing id order makes the order inside a cell the id order. */
static void counting_sort(const or_grid *g, int n, const float *pos3,
                          unsigned *keys, int *perm, int *cell_start)
{
    long nc = g->ncells;
    int *count = (int *)calloc((size_t)nc, sizeof(int));
    int *cursor = (int *)calloc((size_t)nc, sizeof(int));
    for (int i = 0; i < n; ++i) {
        keys[i] = (unsigned)key_of(g, pos3 + 3 * i);
        count[keys[i]] += 1;
    }
    cell_start[0] = 0;
    for (long c = 0; c < nc; ++c) cell_start[c + 1] = cell_start[c] + count[c];
    for (int i = 0; i < n; ++i) {
        unsigned c = keys[i];
        perm[cell_start[c] + cursor[c]] = i;
        cursor[c] += 1;
    }
    free(count);
    free(cursor);
}

/* --------------------------------------------------------- predicates */

/* Squared distance in float32 with the fixed operation order. */
static float r2_f32(const float *xi, const float *xj)
{
    float dx = xj[0] - xi[0];
    float dy = xj[1] - xi[1];
    float dz = xj[2] - xi[2];
    return fmaf(dz, dz, fmaf(dy, dy, dx * dx));
}

/* ----------------------------------------------------------- kernels */

/* poly6 (section "Smoothed Particle Hydrodynamics"): 315/(64 pi h^9) (h^2-r^2)^3. */
static double w_poly6(double h, double r2)
{
    double h2 = h * h;
    if (r2 > h2) return 0.0;
    double t = h2 - r2;
    return 315.0 / (64.0 * OR_PI * pow(h, 9)) * t * t * t;
}

/* Spiky-gradient and viscosity-Laplacian prefactors (section "Pressure and
 * Viscosity"): grad W = -C_p (1-q)^2 / q * r,  lap W = C_v (1-q). */
static void force_constants(const or_params *p, double *cp, double *cv)
{
    double h = p->h;
    if (p->const_set == 1) {           /* as printed: 2-D normalisations */
        *cp = 30.0 / (OR_PI * pow(h, 4));
        *cv = 40.0 / (OR_PI * pow(h, 4));
    } else {                            /* 3-D normalised spiky / viscosity kernels */
        *cp = 45.0 / (OR_PI * pow(h, 5));
        *cv = 45.0 / (OR_PI * pow(h, 5));
    }
}

/* ------------------------------------------------------ neighbour walk */

/* The stencil around the particle's own cell (get_nearby_key: 27 cells for
 * d >= h), out-of-grid cells skipped, visited dz outer, dy, dx inner;
 * particles of a cell in sorted (id) order.  The stencil reaches
 * reach = ceil(h/d) + 1 cells: one more than ceil(h/d), so that a neighbour
 * whose float32 cell index rounded across a cell face is still visited. */
typedef struct {
    const or_grid *g;
    const int *perm, *cell_start;
    int reach, reach_x;     /* along y and z, along x */
} or_walk;

static int walk_reach(double h, double d) { return (int)ceil(h / d) + 1; }

#define FOR_EACH_CANDIDATE(W, XI, J, ...)                                        \
    do {                                                                         \
        int cx_ = cell_coord((W)->g, 0, (XI)[0]);                                \
        int cy_ = cell_coord((W)->g, 1, (XI)[1]);                                \
        int cz_ = cell_coord((W)->g, 2, (XI)[2]);                                \
        const int R_ = (W)->reach, RX_ = (W)->reach_x;                           \
        for (int dz_ = -R_; dz_ <= R_; ++dz_)                                    \
            for (int dy_ = -R_; dy_ <= R_; ++dy_)                                \
                for (int dx_ = -RX_; dx_ <= RX_; ++dx_) {                        \
                    int x_ = cx_ + dx_, y_ = cy_ + dy_, z_ = cz_ + dz_;          \
                    if (x_ < 0 || x_ >= (W)->g->dim[0] || y_ < 0 ||              \
                        y_ >= (W)->g->dim[1] || z_ < 0 || z_ >= (W)->g->dim[2])  \
                        continue;                                                \
                    long c_ = cell_hash((W)->g, x_, y_, z_);                     \
                    for (int s_ = (W)->cell_start[c_];                           \
                         s_ < (W)->cell_start[c_ + 1]; ++s_) {                   \
                        int J = (W)->perm[s_];                                   \
                        __VA_ARGS__                                              \
                    }                                                            \
                }                                                                \
    } while (0)

/* Pair filter: j != i, and no pair of two boid-attached particles. */
static int pair_allowed(int i, int j, int n_att)
{
    return j != i && !(i < n_att && j < n_att);
}

/* ------------------------------------------------------------ exports */

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

int or_grid_dims(const or_params *p, int which, int dims[3])
{
    or_grid g;
    if (which) grid_make(&g, p->box_min, p->box_max, p->boid_cell_size);
    else grid_make_x(&g, p->box_min, p->box_max, cell_x(p), p->cell_size);
    for (int a = 0; a < 3; ++a) dims[a] = g.dim[a];
    return 0;
}

/* Kernel values for the normalisation and derivative pins. */
double or_w_poly6(const or_params *p, double r) { return w_poly6(p->h, r * r); }

/* Scalar s with grad W_spiky(r_vec) = s * r_vec, |r_vec| = r in (0, h). */
double or_grad_spiky_factor(const or_params *p, double r)
{
    double cp, cv, q = r / p->h;
    force_constants(p, &cp, &cv);
    if (r <= 0.0 || q >= 1.0) return 0.0;
    return -cp * (1.0 - q) * (1.0 - q) / q;
}

double or_lap_visc(const or_params *p, double r)
{
    double cp, cv, q = r / p->h;
    force_constants(p, &cp, &cv);
    if (q >= 1.0) return 0.0;
    return cv * (1.0 - q);
}

/* Mass that makes the density of an infinite cubic lattice of the given
 * spacing equal the rest density: m = rho0 / sum_o W(|o| s) over all lattice
 * offsets o (self included) with |o| s < h. */
double or_lattice_mass(const or_params *p, double spacing)
{
    int R = (int)ceil(p->h / spacing) + 1;
    double sum = 0.0;
    for (int z = -R; z <= R; ++z)
        for (int y = -R; y <= R; ++y)
            for (int x = -R; x <= R; ++x) {
                double r2 = ((double)x * x + (double)y * y + (double)z * z) * spacing * spacing;
                if (r2 < p->h * p->h) sum += w_poly6(p->h, r2);
            }
    return p->rho0 / sum;
}

/* The paper's integer hash generator: stream s = seed + id; each draw
 * scrambles s and returns it.  Writes ncalls draws of one stream. */
void or_rng_stream(uint32_t seed, uint32_t id, int ncalls, uint32_t *out)
{
    uint32_t s = seed + id;
    for (int c = 0; c < ncalls; ++c) {
        s ^= 2747636419u;
        s *= 2654435769u;
        s ^= s >> 16;
        s *= 2654435769u;
        s ^= s >> 16;
        s *= 2654435769u;
        out[c] = s;
    }
}

/* Binning alone: keys, sorted permutation, cell_start (ncells + 1). */
int or_bin(const or_params *p, int which, int n, const float *pos3,
           unsigned *keys, int *perm, int *cell_start)
{
    or_grid g;
    if (which) grid_make(&g, p->box_min, p->box_max, p->boid_cell_size);
    else grid_make_x(&g, p->box_min, p->box_max, cell_x(p), p->cell_size);
    counting_sort(&g, n, pos3, keys, perm, cell_start);
    return 0;
}

/* Neighbour sets through the grid, in walk order.  counts[i] = |N(i)|;
 * if offsets/list are given, list[offsets[i] ..] receives the ids of N(i)
 * in the order the 27-cell walk meets them.  N(i) = { j : pair_allowed,
 * r2_f32 < h*h }.  Ids < n_att are boid-attached. */
int or_neighbors(const or_params *p, int n, int n_att, const float *pos3,
                 int *counts, const long *offsets, int *list)
{
    or_grid g;
    grid_make_x(&g, p->box_min, p->box_max, cell_x(p), p->cell_size);
    unsigned *keys = (unsigned *)malloc(sizeof(unsigned) * (size_t)(n > 0 ? n : 1));
    int *perm = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    int *cs = (int *)malloc(sizeof(int) * (size_t)(g.ncells + 1));
    counting_sort(&g, n, pos3, keys, perm, cs);
    or_walk w = {&g, perm, cs, walk_reach(p->h, p->cell_size), walk_reach(p->h, cell_x(p))};
    float hf = (float)p->h, h2f = hf * hf;
#pragma omp parallel for schedule(dynamic, 64)
    for (int i = 0; i < n; ++i) {
        const float *xi = pos3 + 3 * i;
        int c = 0;
        FOR_EACH_CANDIDATE(&w, xi, j, {
            if (pair_allowed(i, j, n_att) && r2_f32(xi, pos3 + 3 * j) < h2f) {
                if (list) list[offsets[i] + c] = j;
                ++c;
            }
        });
        counts[i] = c;
    }
    free(keys); free(perm); free(cs);
    return 0;
}

/* Neighbour sets by brute force over all pairs (no grid), ids ascending. */
int or_brute_neighbors(const or_params *p, int n, int n_att, const float *pos3,
                       int *counts, const long *offsets, int *list)
{
    float hf = (float)p->h, h2f = hf * hf;
#pragma omp parallel for schedule(dynamic, 64)
    for (int i = 0; i < n; ++i) {
        int c = 0;
        for (int j = 0; j < n; ++j)
            if (pair_allowed(i, j, n_att) && r2_f32(pos3 + 3 * i, pos3 + 3 * j) < h2f) {
                if (list) list[offsets[i] + c] = j;
                ++c;
            }
        counts[i] = c;
    }
    return 0;
}

/* f_ij of the symmetrised pressure force and the velocity-difference
 * viscosity force (section "Pressure and Viscosity"), with
 * r_ij = x_i - x_j, v_ij = v_i - v_j, q = |r_ij| / h:
 *   f_ij = m/rho_j * [ C_p (p_i + p_j)/2 (1-q)^2/q r_ij - C_v mu (1-q) v_ij ]
 * Returns 0 for r2 >= h^2 or r2 == 0 (listing "Compute acceleration").
 *
 * abs_out receives the error scale of a float32 evaluation of f_ij: for each
 * term its magnitude plus r^2 |d(term)/d(r^2)|, the forward-error factor of a
 * relative rounding of the float32 squared distance (1 - q cancels near the
 * kernel's edge), with the equation-of-state sum taken as (|p_i| + |p_j|)/2
 * (it cancels where rho_i < rho0 < rho_j):
 *   m/rho_j [ C_p (|p_i| + |p_j|)/2 h (1-q) + C_v mu |v_ij| (1 - q/2) ]. */
static void pair_force(const or_params *p, double cp, double cv,
                       const double *xi, const double *xj,
                       const double *vi, const double *vj,
                       double rho_i, double rho_j, double f[3], double *abs_out)
{
    double r[3] = {xi[0] - xj[0], xi[1] - xj[1], xi[2] - xj[2]};
    double v[3] = {vi[0] - vj[0], vi[1] - vj[1], vi[2] - vj[2]};
    double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
    f[0] = f[1] = f[2] = 0.0;
    *abs_out = 0.0;
    if (r2 == 0.0 || r2 >= p->h * p->h) return;
    double q = sqrt(r2) / p->h;
    double pi = p->k * (rho_i - p->rho0);   /* equation of state p = k (rho - rho0) */
    double pj = p->k * (rho_j - p->rho0);
    double pres = cp * 0.5 * (pi + pj) * (1.0 - q) * (1.0 - q) / q;
    double visc = cv * p->mu * (1.0 - q);
    for (int a = 0; a < 3; ++a) f[a] = p->mass / rho_j * (pres * r[a] - visc * v[a]);
    double vmag = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    *abs_out = p->mass / rho_j * (cp * 0.5 * (fabs(pi) + fabs(pj)) * p->h * (1.0 - q) +
                                  cv * p->mu * vmag * (1.0 - 0.5 * q));
}

/* ----------------------------------------------------- obstacle grid */

/* Centre of boid-grid cell i along axis a: fl(min + fl(fl(i + 0.5) d)). */
static float cell_centre(const or_params *p, int a, int i)
{
    const float d = (float)p->boid_cell_size;
    return (float)p->box_min[a] + ((float)i + 0.5f) * d;
}

/* The obstacle grid (the boid grid's cells): every obstacle whose surface
 * passes within half a cell diagonal of a cell's centre (|sdf| <= fl(0.8660254 d),
 * the signed distance evaluated in float32 in a fixed order) adds its
 * outward unit normal at the surface point nearest the centre; the cell
 * keeps the mean of those normals and their count: out4[4 c + 0..2] = mean
 * normal, out4[4 c + 3] = count.  Reading: spheres and boxes stand in for
 * the paper's meshes, whose normals it attributes to grid cells. */
int or_obstacle_grid(const or_params *p, const or_obstacles *ob, double *out4)
{
    or_grid g;
    grid_make(&g, p->box_min, p->box_max, p->boid_cell_size);
    const float half_diag = 0.866025403784f * (float)p->boid_cell_size;
    for (long c = 0; c < g.ncells; ++c) {
        const int ix = (int)(c % g.dim[0]), iy = (int)((c / g.dim[0]) % g.dim[1]),
                  iz = (int)(c / ((long)g.dim[0] * g.dim[1]));
        const float x[3] = {cell_centre(p, 0, ix), cell_centre(p, 1, iy), cell_centre(p, 2, iz)};
        double sum[3] = {0, 0, 0};
        int cnt = 0;
        for (int k = 0; ob && k < ob->n_sphere; ++k) {
            const float *S = ob->sphere + 4 * k;
            const float d[3] = {x[0] - S[0], x[1] - S[1], x[2] - S[2]};
            const float q2 = fmaf(d[2], d[2], fmaf(d[1], d[1], d[0] * d[0]));
            const float dist = sqrtf(q2) - S[3];
            if (!(fabsf(dist) <= half_diag) || !(q2 > 0.0f)) continue;
            const double len = sqrt((double)d[0] * d[0] + (double)d[1] * d[1] + (double)d[2] * d[2]);
            for (int a = 0; a < 3; ++a) sum[a] += d[a] / len;
            ++cnt;
        }
        for (int k = 0; ob && k < ob->n_box; ++k) {
            const float *B = ob->box + 6 * k;
            float q[3], m[3];
            for (int a = 0; a < 3; ++a) {
                q[a] = fmaxf(B[a] - x[a], x[a] - B[3 + a]);
                m[a] = fmaxf(q[a], 0.0f);
            }
            const int outside = q[0] > 0.0f || q[1] > 0.0f || q[2] > 0.0f;
            const float dist = outside ? sqrtf(fmaf(m[2], m[2], fmaf(m[1], m[1], m[0] * m[0])))
                                       : fmaxf(q[0], fmaxf(q[1], q[2]));
            if (!(fabsf(dist) <= half_diag)) continue;
            double n[3] = {0, 0, 0};
            if (outside) {
                double len = 0.0;
                for (int a = 0; a < 3; ++a) {
                    n[a] = x[a] > B[3 + a] ? (double)m[a] : (x[a] < B[a] ? -(double)m[a] : 0.0);
                    len += n[a] * n[a];
                }
                len = sqrt(len);
                for (int a = 0; a < 3; ++a) n[a] /= len;
            } else {
                int ax = 0;  /* the nearest face: largest q, the lowest axis on ties */
                for (int a = 1; a < 3; ++a)
                    if (q[a] > q[ax]) ax = a;
                n[ax] = (x[ax] - B[3 + ax] >= B[ax] - x[ax]) ? 1.0 : -1.0;
            }
            for (int a = 0; a < 3; ++a) sum[a] += n[a];
            ++cnt;
        }
        for (int a = 0; a < 3; ++a) out4[4 * c + a] = cnt ? sum[a] / cnt : 0.0;
        out4[4 * c + 3] = cnt;
    }
    return 0;
}

/* Obstacle avoidance of a boid at pb (section "Boid Motion and Agent Fluid
 * Interaction"): the mean over the obstacle cells whose centre lies within
 * the visual range (float32 predicate as the boid pairs) of their mean
 * normals, those within the protection range weighted near_factor;
 * returns the count and the increment w_obst * that mean in dv. */
static int obstacle_term(const or_params *p, const or_obstacles *ob, const or_grid *g, const double *grid4,
                         const float *pb, float rs2f, float rv2f, double dv[3])
{
    double acc[3] = {0, 0, 0};
    int n = 0;
    for (long c = 0; c < g->ncells; ++c) {
        if (grid4[4 * c + 3] == 0.0) continue;
        const int ix = (int)(c % g->dim[0]), iy = (int)((c / g->dim[0]) % g->dim[1]),
                  iz = (int)(c / ((long)g->dim[0] * g->dim[1]));
        const float x[3] = {cell_centre(p, 0, ix), cell_centre(p, 1, iy), cell_centre(p, 2, iz)};
        const float r2 = r2_f32(pb, x);
        if (!(r2 < rv2f)) continue;
        const double w = r2 < rs2f ? ob->near_factor : 1.0;
        for (int a = 0; a < 3; ++a) acc[a] += w * grid4[4 * c + a];
        ++n;
    }
    for (int a = 0; a < 3; ++a) dv[a] = n ? ob->w_obst * acc[a] / n : 0.0;
    return n;
}

int or_step(const or_params *p, int n_fluid, int n_boid,
            const float *fluid_pos, const float *fluid_vel,
            const float *boid_pos, const float *boid_vel, or_outputs *out)
{
    if (p->coupling_mode != 0 && p->coupling_mode != 1) return -1;
    const int literal = p->coupling_mode == 1;
    const int nb = n_boid, n = n_fluid + n_boid;
    or_grid g;
    grid_make_x(&g, p->box_min, p->box_max, cell_x(p), p->cell_size);

    /* 1. attach a particle to every boid: the boid's position; its velocity
     *    is the boid's (force coupling) or the attached particle's own,
     *    carried from the previous step (literal coupling). */
    float *x32 = (float *)malloc(sizeof(float) * 3 * (size_t)(n > 0 ? n : 1));
    double *x = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    double *v = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    for (int b = 0; b < nb; ++b)
        for (int a = 0; a < 3; ++a) {
            x32[3 * b + a] = boid_pos[3 * b + a];
            v[3 * b + a] = literal && p->att_vel ? p->att_vel[3 * b + a] : boid_vel[3 * b + a];
        }
    for (int f = 0; f < n_fluid; ++f)
        for (int a = 0; a < 3; ++a) {
            x32[3 * (nb + f) + a] = fluid_pos[3 * f + a];
            v[3 * (nb + f) + a] = fluid_vel[3 * f + a];
        }
    for (int i = 0; i < 3 * n; ++i) x[i] = x32[i];

    /* 2. binning. */
    unsigned *keys = (unsigned *)malloc(sizeof(unsigned) * (size_t)(n > 0 ? n : 1));
    int *perm = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    int *cs = (int *)malloc(sizeof(int) * (size_t)(g.ncells + 1));
    counting_sort(&g, n, x32, keys, perm, cs);
    or_walk w = {&g, perm, cs, walk_reach(p->h, p->cell_size), walk_reach(p->h, cell_x(p))};
    float hf = (float)p->h, h2f = hf * hf;

    /* 3. density (self term included) and pressure. */
    double *rho = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
#pragma omp parallel for schedule(dynamic, 64)
    for (int i = 0; i < n; ++i) {
        const float *xi = x32 + 3 * i;
        double sum = w_poly6(p->h, 0.0);
        int cnt = 0;
        FOR_EACH_CANDIDATE(&w, xi, j, {
            if (pair_allowed(i, j, nb) && r2_f32(xi, x32 + 3 * j) < h2f) {
                double dx = x[3 * j] - x[3 * i], dy = x[3 * j + 1] - x[3 * i + 1],
                       dz = x[3 * j + 2] - x[3 * i + 2];
                sum += w_poly6(p->h, dx * dx + dy * dy + dz * dz);
                ++cnt;
            }
        });
        rho[i] = p->mass * sum;
        if (out->nbr_count) out->nbr_count[i] = cnt;
    }

    /* 4. accelerations: a_i = (1/rho_i) sum_j f_ij (+ g for fluid). */
    double cp, cv;
    force_constants(p, &cp, &cv);
    double *acc = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    double gnorm = sqrt(p->g[0] * p->g[0] + p->g[1] * p->g[1] + p->g[2] * p->g[2]);
#pragma omp parallel for schedule(dynamic, 64)
    for (int i = 0; i < n; ++i) {
        const float *xi = x32 + 3 * i;
        double sum[3] = {0, 0, 0}, infl[3] = {0, 0, 0}, abs_sum = 0.0;
        int touched = 0;
        FOR_EACH_CANDIDATE(&w, xi, j, {
            if (pair_allowed(i, j, nb) && r2_f32(xi, x32 + 3 * j) < h2f) {
                double f[3], fa;
                pair_force(p, cp, cv, x + 3 * i, x + 3 * j, v + 3 * i, v + 3 * j,
                           rho[i], rho[j], f, &fa);
                for (int a = 0; a < 3; ++a) sum[a] += f[a];
                abs_sum += fa;
                if (j < nb && (x[3 * i] != x[3 * j] || x[3 * i + 1] != x[3 * j + 1] ||
                               x[3 * i + 2] != x[3 * j + 2])) {
                    ++touched;                      /* touched_by_boid */
                    for (int a = 0; a < 3; ++a) infl[a] += f[a];
                }
            }
        });
        int fluid = i >= nb;
        for (int a = 0; a < 3; ++a) acc[3 * i + a] = sum[a] / rho[i] + (fluid ? p->g[a] : 0.0);
        if (out->acc_scale) out->acc_scale[i] = abs_sum / rho[i] + (fluid ? gnorm : 0.0);
        if (out->touched) out->touched[i] = touched;
        if (out->influence)
            for (int a = 0; a < 3; ++a) out->influence[3 * i + a] = infl[a] / rho[i];
    }

    /* 5. boid rules on the start-of-step snapshot (brute force over boids). */
    float rs = (float)p->r_sep, rv = (float)p->r_vis;
    float rs2f = rs * rs, rv2f = rv * rv;
    const or_obstacles *ob = (const or_obstacles *)p->obstacles;
    or_grid gob;
    double *grid4 = NULL;
    if (ob) {
        grid_make(&gob, p->box_min, p->box_max, p->boid_cell_size);
        grid4 = (double *)calloc((size_t)gob.ncells * 4, sizeof(double));
        or_obstacle_grid(p, ob, grid4);
    }
    for (int b = 0; b < nb; ++b) {
        const float *pb = boid_pos + 3 * b;
        double vb[3] = {boid_vel[3 * b], boid_vel[3 * b + 1], boid_vel[3 * b + 2]};
        double pbd[3] = {pb[0], pb[1], pb[2]};
        double close[3] = {0, 0, 0}, close_abs = 0.0;
        double va[3] = {0, 0, 0}, pa[3] = {0, 0, 0};
        int nsep = 0, nvis = 0;
        for (int j = 0; j < nb; ++j) {
            if (j == b) continue;
            const float *pj = boid_pos + 3 * j;
            float r2 = r2_f32(pb, pj);
            double d[3] = {pbd[0] - pj[0], pbd[1] - pj[1], pbd[2] - pj[2]};
            if (r2 < rs2f) {                         /* separation: inside protect range */
                double len = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                double wgt = 1.0 - len / p->r_sep;
                wgt = wgt < 0.0 ? 0.0 : (wgt > 1.0 ? 1.0 : wgt);
                for (int a = 0; a < 3; ++a) close[a] += d[a] * wgt;
                close_abs += len * wgt;
                ++nsep;
            }
            if (r2 < rv2f) {                         /* alignment / cohesion: visual range */
                for (int a = 0; a < 3; ++a) {
                    va[a] += boid_vel[3 * j + a];
                    pa[a] += pj[a];
                }
                ++nvis;
            }
        }
        double scale = sqrt(vb[0] * vb[0] + vb[1] * vb[1] + vb[2] * vb[2]);
        for (int a = 0; a < 3; ++a) vb[a] += p->w_sep * close[a];
        scale += p->w_sep * close_abs;
        if (nvis > 0) {
            double vam = 0, vn = 0;
            for (int a = 0; a < 3; ++a) va[a] /= nvis;
            for (int a = 0; a < 3; ++a) { vam += va[a] * va[a]; vn += vb[a] * vb[a]; }
            for (int a = 0; a < 3; ++a) vb[a] += p->w_align * (va[a] - vb[a]);
            scale += p->w_align * (sqrt(vam) + sqrt(vn));
            double pam = 0, pn = 0;
            for (int a = 0; a < 3; ++a) pa[a] /= nvis;
            for (int a = 0; a < 3; ++a) { pam += pa[a] * pa[a]; pn += pbd[a] * pbd[a]; }
            for (int a = 0; a < 3; ++a) vb[a] += p->w_coh * (pa[a] - pbd[a]);
            scale += p->w_coh * (sqrt(pam) + sqrt(pn));
        }
        double vatt[3] = {0.0, 0.0, 0.0};
        if (literal) {
            /* literal coupling (section "Boid Motion and Agent Fluid
             * Interaction", the velocity update with sph_factor): the
             * attached particle is integrated like every particle, gravity
             * included (the frame loop integrates all particles before the
             * boid pass), and the boid adds sph_factor times its velocity */
            double vs = 0.0;
            for (int a = 0; a < 3; ++a) {
                vatt[a] = v[3 * b + a] + p->dt * (acc[3 * b + a] + p->g[a]);
                vb[a] += p->sph_factor * vatt[a];
                vs += v[3 * b + a] * v[3 * b + a];
            }
            if (out->acc_scale) scale += fabs(p->sph_factor) * (sqrt(vs) + p->dt * (out->acc_scale[b] + gnorm));
        } else {
            /* fluid -> boid: v += sph_factor * dt * F_b, F_b the attached particle's acceleration */
            for (int a = 0; a < 3; ++a) vb[a] += p->sph_factor * p->dt * acc[3 * b + a];
            if (out->acc_scale) scale += fabs(p->sph_factor) * p->dt * out->acc_scale[b];
        }
        /* obstacle avoidance (reading: after the fluid coupling, before the
         * edge avoidance and the speed limit, which still bound the result) */
        if (ob) {
            double dv[3];
            obstacle_term(p, ob, &gob, grid4, pb, rs2f, rv2f, dv);
            for (int a = 0; a < 3; ++a) vb[a] += dv[a];
            scale += fabs(ob->w_obst) * (ob->near_factor > 1.0 ? ob->near_factor : 1.0);
        }
        /* edge avoidance: steer back into the box */
        for (int a = 0; a < 3; ++a) {
            if (pb[a] < (float)p->box_min[a]) vb[a] += p->edge_turn;
            if (pb[a] > (float)p->box_max[a]) vb[a] -= p->edge_turn;
        }
        scale += 3.0 * p->edge_turn;
        /* speed limit */
        double sp = sqrt(vb[0] * vb[0] + vb[1] * vb[1] + vb[2] * vb[2]);
        if (sp > p->v_max) {
            for (int a = 0; a < 3; ++a) vb[a] *= p->v_max / sp;
        } else if (sp > 0.0 && sp < p->v_min) {
            for (int a = 0; a < 3; ++a) vb[a] *= p->v_min / sp;
        }
        if (out->new_boid_vel) for (int a = 0; a < 3; ++a) out->new_boid_vel[3 * b + a] = vb[a];
        /* the attached particle follows the boid's position into the next
         * step; its velocity is the boid's (force) or its own (literal) */
        if (out->new_att_vel) for (int a = 0; a < 3; ++a) out->new_att_vel[3 * b + a] = literal ? vatt[a] : vb[a];
        if (out->new_boid_pos)
            for (int a = 0; a < 3; ++a) out->new_boid_pos[3 * b + a] = pbd[a] + vb[a] * p->dt;
        if (out->boid_vscale) out->boid_vscale[b] = scale;
        if (out->boid_nsep) out->boid_nsep[b] = nsep;
        if (out->boid_nvis) out->boid_nvis[b] = nvis;
        if (out->fb) for (int a = 0; a < 3; ++a) out->fb[3 * b + a] = acc[3 * b + a];
    }

    free(grid4);

    /* 6. Euler-Cromer for fluid particles, then damped reflection at the walls. */
    for (int f = 0; f < n_fluid; ++f) {
        int i = nb + f;
        double vn[3], xn[3], margin = INFINITY;
        for (int a = 0; a < 3; ++a) {
            vn[a] = v[3 * i + a] + acc[3 * i + a] * p->dt;
            xn[a] = x[3 * i + a] + vn[a] * p->dt;
        }
        if (out->pre_wall_pos) for (int a = 0; a < 3; ++a) out->pre_wall_pos[3 * f + a] = xn[a];
        if (out->pre_wall_vel) for (int a = 0; a < 3; ++a) out->pre_wall_vel[3 * f + a] = vn[a];
        for (int a = 0; a < 3; ++a) {
            double lo = p->box_min[a], hi = p->box_max[a];
            double m1 = fabs(xn[a] - lo), m2 = fabs(xn[a] - hi);
            margin = fmin(margin, fmin(m1, m2));
            if (xn[a] < lo) {
                xn[a] = 2.0 * lo - xn[a];
                vn[a] = -p->wall_restitution * vn[a];
            } else if (xn[a] > hi) {
                xn[a] = 2.0 * hi - xn[a];
                vn[a] = -p->wall_restitution * vn[a];
            }
            if (xn[a] < lo) xn[a] = lo;
            if (xn[a] > hi) xn[a] = hi;
        }
        if (out->wall_margin) out->wall_margin[f] = margin;
        if (out->new_fluid_pos) for (int a = 0; a < 3; ++a) out->new_fluid_pos[3 * f + a] = xn[a];
        if (out->new_fluid_vel) for (int a = 0; a < 3; ++a) out->new_fluid_vel[3 * f + a] = vn[a];
    }

    /* outputs of the intermediate passes */
    for (int i = 0; i < n; ++i) {
        if (out->rho) out->rho[i] = rho[i];
        if (out->pressure) out->pressure[i] = p->k * (rho[i] - p->rho0);
        if (out->acc) for (int a = 0; a < 3; ++a) out->acc[3 * i + a] = acc[3 * i + a];
        if (out->keys) out->keys[i] = keys[i];
        if (out->perm) out->perm[i] = perm[i];
    }
    if (out->cell_start) memcpy(out->cell_start, cs, sizeof(int) * (size_t)(g.ncells + 1));
    if (out->boid_keys || out->boid_perm || out->boid_cell_start) {
        or_grid gb;
        grid_make(&gb, p->box_min, p->box_max, p->boid_cell_size);
        unsigned *bk = (unsigned *)malloc(sizeof(unsigned) * (size_t)(nb > 0 ? nb : 1));
        int *bp = (int *)malloc(sizeof(int) * (size_t)(nb > 0 ? nb : 1));
        int *bc = (int *)malloc(sizeof(int) * (size_t)(gb.ncells + 1));
        counting_sort(&gb, nb, boid_pos, bk, bp, bc);
        if (out->boid_keys) memcpy(out->boid_keys, bk, sizeof(unsigned) * (size_t)nb);
        if (out->boid_perm) memcpy(out->boid_perm, bp, sizeof(int) * (size_t)nb);
        if (out->boid_cell_start) memcpy(out->boid_cell_start, bc, sizeof(int) * (size_t)(gb.ncells + 1));
        free(bk); free(bp); free(bc);
    }
    free(x32); free(x); free(v); free(keys); free(perm); free(cs); free(rho); free(acc);
    return 0;
}

/* ------------------------------------------------------ voxel density */

/* Voxel density (section "Voxel Density") at every corner of a grid:
 *   phi(x) = |x - xbar| - rbar,  xbar = sum_i w_i x_i,  rbar = r,
 *   w_i = k(|x - x_i| / R) / sum_j k(|x - x_j| / R),  k(s) = (1 - s^2)^3,
 * over the n particles pos3 with |x - x_i| < R, the distance decided in
 * float32 like the step's neighbour predicate (d = x_i - x per component,
 * r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx)) < fl(R * R)).  Corner
 * (ix, iy, iz) is at fl(origin + fl(i * spacing)) per axis and has index
 * ix + nx (iy + ny iz).  A corner without neighbours gets phi = R.  The
 * candidates come from a plain grid of cell R over the particles' bounding
 * box, two cells each way (a candidate list, not a result: the predicate
 * decides).  Values in double.  Returns 0, or -1 on bad arguments. */
int or_voxel_density(int n, const float *pos3, const float *origin, float spacing, const int *dims,
                     float radius, float particle_radius, double *phi, int *count)
{
    if (n < 0 || !origin || !dims || !phi || spacing <= 0.0f || radius <= 0.0f) return -1;
    const float R2 = radius * radius;
    double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    for (int a = 0; a < 3; ++a) {
        lo[a] = 1e300;
        hi[a] = -1e300;
    }
    for (int i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) {
            if (pos3[3 * i + a] < lo[a]) lo[a] = pos3[3 * i + a];
            if (pos3[3 * i + a] > hi[a]) hi[a] = pos3[3 * i + a];
        }
    int gd[3] = {1, 1, 1};
    if (n > 0)
        for (int a = 0; a < 3; ++a) gd[a] = (int)floor((hi[a] - lo[a]) / radius) + 1;
    long gcells = (long)gd[0] * gd[1] * gd[2];
    int *gstart = (int *)calloc((size_t)gcells + 1, sizeof(int));
    int *gidx = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    int *gcell = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) {
        int c[3];
        for (int a = 0; a < 3; ++a) {
            c[a] = (int)floor((pos3[3 * i + a] - lo[a]) / radius);
            if (c[a] < 0) c[a] = 0;
            if (c[a] >= gd[a]) c[a] = gd[a] - 1;
        }
        gcell[i] = c[0] + gd[0] * (c[1] + gd[1] * c[2]);
        gstart[gcell[i] + 1] += 1;
    }
    for (long c = 0; c < gcells; ++c) gstart[c + 1] += gstart[c];
    int *cur = (int *)calloc((size_t)gcells, sizeof(int));
    for (int i = 0; i < n; ++i) gidx[gstart[gcell[i]] + cur[gcell[i]]++] = i;
    free(cur);
    const long ncorner = (long)dims[0] * dims[1] * dims[2];
#pragma omp parallel for schedule(dynamic, 256)
    for (long idx = 0; idx < ncorner; ++idx) {
        const int ix = (int)(idx % dims[0]), iy = (int)((idx / dims[0]) % dims[1]),
                  iz = (int)(idx / ((long)dims[0] * dims[1]));
        float x[3];
        x[0] = origin[0] + (float)ix * spacing;
        x[1] = origin[1] + (float)iy * spacing;
        x[2] = origin[2] + (float)iz * spacing;
        int c[3];
        for (int a = 0; a < 3; ++a) c[a] = (int)floor((x[a] - lo[a]) / radius);
        double ksum = 0.0, kx[3] = {0, 0, 0};
        int cnt = 0;
        for (int z = c[2] - 2; z <= c[2] + 2; ++z)
            for (int y = c[1] - 2; y <= c[1] + 2; ++y)
                for (int xx = c[0] - 2; xx <= c[0] + 2; ++xx) {
                    if (xx < 0 || y < 0 || z < 0 || xx >= gd[0] || y >= gd[1] || z >= gd[2]) continue;
                    const long g = xx + (long)gd[0] * (y + (long)gd[1] * z);
                    for (int k = gstart[g]; k < gstart[g + 1]; ++k) {
                        const float *p = pos3 + 3 * gidx[k];
                        if (!(r2_f32(x, p) < R2)) continue;
                        double d2 = 0.0;
                        for (int a = 0; a < 3; ++a) d2 += ((double)p[a] - x[a]) * ((double)p[a] - x[a]);
                        const double s2 = d2 / ((double)radius * radius);
                        const double w = (1.0 - s2) * (1.0 - s2) * (1.0 - s2);
                        ksum += w;
                        for (int a = 0; a < 3; ++a) kx[a] += w * p[a];
                        ++cnt;
                    }
                }
        if (count) count[idx] = cnt;
        if (cnt == 0) {
            phi[idx] = radius;
            continue;
        }
        double dist2 = 0.0;
        for (int a = 0; a < 3; ++a) {
            const double xb = kx[a] / ksum;
            dist2 += (x[a] - xb) * (x[a] - xb);
        }
        phi[idx] = sqrt(dist2) - (double)particle_radius;
    }
    free(gstart);
    free(gidx);
    free(gcell);
    return 0;
}
