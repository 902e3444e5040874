// sph_internal.cuh -- device helpers, per-step constants and the handle of the
// GB300 SPH-with-boids step library.  Everything here is internal; the public
// surface is include/sph.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sph.h"

namespace sphk {

constexpr unsigned FULL = 0xffffffffu;

// Bounds checks of the bounds-checked build (compiled with -DSPH_CHECK, a
// stand-in for a memory sanitizer): an index i outside [0, n) sets
// SPH_DEV_BOUNDS in the error word and the access is skipped.  In the
// normal build the check compiles to nothing.
#ifdef SPH_CHECK
#define SPH_IN_BOUNDS(i, n, err) \
    ((unsigned)(i) < (unsigned)(n) ? true : (atomicOr((err), SPH_DEV_BOUNDS), false))
#else
#define SPH_IN_BOUNDS(i, n, err) true
#endif

// A uniform grid over the box (section "Neighborhood Search"): dim cells per
// axis, float32 origin and reciprocal cell sizes used by get_cell (inv_dx
// along x, inv_d along y and z; equal unless the cells are made narrower
// along x, the axis along which a row of cells is one contiguous run of
// sorted slots).
struct GridDesc {
    int dim[3];
    int ncells;
    float minf[3];
    float inv_d;
    float inv_dx;
};

// Conservative search bounds of a grid walk: any particle j with
// pair_r2 < r2_bound lies within `reach` of the query along every axis and
// within `reach2` in squared distance; `margin` covers the float32
// rounding of cell boundaries (cell = floor((p - m) * inv_d)).
struct WalkBounds {
    float reach2;   // r2_bound * (1 + 1e-5)
    float reach;    // sqrt(reach2) + margin
    float margin;   // absolute slack on cell boundaries
    float d;        // cell size
};

// Everything a kernel of the step needs about one scene, precomputed on
// the host.  A handle holds one StepConst per scene (a single scene is a
// batch of one).  The scenes' particles, boids and cells occupy consecutive
// ranges of the handle's arrays: scene k owns sorted slots [p_base,
// p_base + n), boids [b_base, b_base + nb), particle cells [c_base, c_base +
// g.ncells) and boid cells [cb_base, cb_base + gb.ncells).  Particle ids are
// global: the attached particle of (global) boid b has id b, fluid particle f
// (global, scene-major) has id nb_all + f, so "attached" is id < nb_all in
// every scene and the order of ids inside a scene is the scene's own order.
struct StepConst {
    GridDesc g;         // particle grid (cell_size)
    GridDesc gb;        // boid grid (boid_cell_size)
    WalkBounds wg;      // particle grid, radius h
    WalkBounds wb;      // boid grid, radius r_vis
    int n;              // particles of the scene: attached + fluid
    int nb;             // boids of the scene
    int nb_all;         // boids of every scene: ids below it are attached
    int p_base, b_base, c_base, cb_base;
    float h2;           // fl(h * h): the neighbour predicate bound
    float mC6;          // m * 315 / (64 pi h^9): poly6 prefactor times mass
    float half_cp_h;    // C_p h / 2: pressure pair prefactor (times 1/r)
    float cv_mu;        // C_v mu: viscosity pair prefactor
    float h, inv_h, mass, k, rho0, dt;  // inv_h = fl(1 / h) (double quotient rounded)
    float grav[3];      // gravity
    float box_min[3], box_max[3];
    float restitution;
    float rs, rs2, rv2; // boid radii (separation) and squared radii
    float w_sep, w_align, w_coh, sph_dt, v_min, v_max, edge_turn;
    float sph_factor;
    int literal;
    // the surrogate's feature grid (cells of h anchored at box_min, cell
    // floor((x - m) inv_h), two cells of margin on every side): dims, and
    // the scene's first cell in the handle's feature grid
    int fdim[3], fc_base;        // SPH_COUPLE_LITERAL: the attached particles keep and integrate their own velocity
    // obstacle avoidance (sph_set_obstacles): off while obst_on == 0
    int obst_on, obst_reach;  // reach: boid-grid cells searched each way
    float w_obst, obst_near;  // gain, weight of cells in the protection range
};

// get_cell along one axis: floor((p - m) * inv_d) in float32, no contraction,
// clamped into [0, dim - 1] (NaN maps to 0).
__device__ __forceinline__ int cell_coord(float x, float mn, float inv_d, int dim, bool* clamped)
{
    float t = __fmul_rn(__fsub_rn(x, mn), inv_d);
    float c = floorf(t);
    if (!(c >= 0.0f)) { *clamped = true; return 0; }
    if (c > (float)(dim - 1)) { *clamped = true; return dim - 1; }
    return (int)c;
}

// hash(c) = c_x + dim_x (c_y + dim_y c_z).
__device__ __forceinline__ unsigned cell_key(const GridDesc& g, float x, float y, float z, bool* clamped)
{
    int cx = cell_coord(x, g.minf[0], g.inv_dx, g.dim[0], clamped);
    int cy = cell_coord(y, g.minf[1], g.inv_d, g.dim[1], clamped);
    int cz = cell_coord(z, g.minf[2], g.inv_d, g.dim[2], clamped);
    return (unsigned)cx + (unsigned)g.dim[0] * ((unsigned)cy + (unsigned)g.dim[1] * (unsigned)cz);
}

// Squared distance of the neighbour predicate: dx = x_j - x_i per component,
// r2 = fma(dz, dz, fma(dy, dy, dx * dx)), every operation rounded once.
__device__ __forceinline__ float pair_r2(float dx, float dy, float dz)
{
    return __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
}

// Warp-aggregated counter increment: lanes with the same key share one
// atomicAdd; returns each lane's slot.  Every lane of the warp must call it.
__device__ __forceinline__ unsigned agg_increment(unsigned* count, unsigned k, bool active)
{
    unsigned act = __ballot_sync(FULL, active);
    unsigned slot = 0;
    if (active) {
        unsigned peers = __match_any_sync(act, k);
        int lane = threadIdx.x & 31;
        int leader = __ffs(peers) - 1;
        unsigned base = 0;
        if (lane == leader) base = atomicAdd(&count[k], (unsigned)__popc(peers));
        base = __shfl_sync(peers, base, leader);
        slot = base + (unsigned)__popc(peers & ((1u << lane) - 1u));
    }
    return slot;
}

__device__ __forceinline__ int id_of(const float4& p) { return __float_as_int(p.w); }

// A fluid position outside the tank [box_min, box_max] (or not a number):
// binning it clamps its cell into the grid, which SPH_DEV_CLAMPED reports.
// Positions on the box faces are inside (their cell may still round onto
// the last grid cell, which is no anomaly).
template <class C>
__device__ __forceinline__ bool outside_box(const C& c, float x, float y, float z)
{
    return !(x >= c.box_min[0] && x <= c.box_max[0] && y >= c.box_min[1] && y <= c.box_max[1] &&
             z >= c.box_min[2] && z <= c.box_max[2]);
}

// Scene of element i: the k with base[k] <= i < base[k + 1] (base has S + 1
// non-decreasing entries, base[0] = 0).  Empty scenes are skipped.
__device__ __forceinline__ int scene_of(const unsigned* __restrict__ base, int S, unsigned i)
{
    int lo = 0, hi = S;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(base + mid) <= i) lo = mid;
        else hi = mid;
    }
    return lo;
}

// The scene table a kernel receives: per-scene constants and the slot /
// boid bases of the scenes.
struct Scenes {
    const StepConst* __restrict__ c;
    const unsigned* __restrict__ pbase;  // S + 1 sorted-slot bases
    const unsigned* __restrict__ bbase;  // S + 1 boid bases
    int S;
    int n_all, nb_all;                   // particles and boids of every scene
};

// Squared distance from v to the padded extent of cell c along one axis;
// the outermost cells of the grid are open towards the outside (positions
// beyond the grid are clamped into them).
__device__ __forceinline__ float axis_gap2(float v, int c, int dim, float mn, const WalkBounds& w)
{
    float lo = c > 0 ? fmaf((float)c, w.d, mn) - w.margin : -INFINITY;
    float hi = c < dim - 1 ? fmaf((float)(c + 1), w.d, mn) + w.margin : INFINITY;
    float gap = fmaxf(0.0f, fmaxf(lo - v, v - hi));
    return gap * gap;
}

// Walk of every cell that can hold a particle within the bound radius of
// (px, py, pz), as rows of contiguous sorted slots: z ascending, then y,
// then the x-cells of the row ascending (the order of the 27-cell walk of
// section "Neighborhood Search", restricted to the cells the sphere can
// reach).  Rows and x-ranges are pruned per query with bounds that are
// conservative for the float32 predicate, so the visited set always holds
// every neighbour.  Usage: RowWalk w(...); while (w.next(s0, s1)) {...}
// yields each non-empty row [s0, s1).
struct RowWalk {
    const GridDesc& g;
    const WalkBounds& wb;
    const unsigned* __restrict__ start;
    float px, py, pz, rz;
    int z, z1, y, y0, y1;

    __device__ __forceinline__ RowWalk(const GridDesc& g_, const WalkBounds& w_, const unsigned* __restrict__ st,
                                       float x_, float y_, float z_)
        : g(g_), wb(w_), start(st), px(x_), py(y_), pz(z_), rz(0.0f)
    {
        bool cl = false;
        const int z0 = cell_coord(pz - wb.reach, g.minf[2], g.inv_d, g.dim[2], &cl);
        z1 = cell_coord(pz + wb.reach, g.minf[2], g.inv_d, g.dim[2], &cl);
        y0 = cell_coord(py - wb.reach, g.minf[1], g.inv_d, g.dim[1], &cl);
        y1 = cell_coord(py + wb.reach, g.minf[1], g.inv_d, g.dim[1], &cl);
        z = z0 - 1;
        y = y1 + 1;  // forces the first next() to open row z0
    }

    __device__ __forceinline__ bool next(unsigned& s0, unsigned& s1)
    {
        for (;;) {
            if (y > y1) {
                if (++z > z1) return false;
                y = y0;
                rz = wb.reach2 - axis_gap2(pz, z, g.dim[2], g.minf[2], wb);
                if (!(rz > 0.0f)) {
                    y = y1 + 1;
                    continue;
                }
            }
            const int yy = y++;
            const float ryz = rz - axis_gap2(py, yy, g.dim[1], g.minf[1], wb);
            if (!(ryz > 0.0f)) continue;
            // x half-width of the row: ryz * rsqrt(ryz) is within 3e-7 of
            // sqrt(ryz) relatively, far inside margin (>= 1e-5 d, d >= h/4)
            const float xr = fmaf(ryz, rsqrtf(ryz), wb.margin);
            bool cl = false;
            const int x0 = cell_coord(px - xr, g.minf[0], g.inv_dx, g.dim[0], &cl);
            const int x1 = cell_coord(px + xr, g.minf[0], g.inv_dx, g.dim[0], &cl);
            const unsigned rowk = (unsigned)g.dim[0] * ((unsigned)yy + (unsigned)g.dim[1] * (unsigned)z);
            s0 = __ldg(start + rowk + x0);
            s1 = __ldg(start + rowk + x1 + 1);
            if (s0 < s1) return true;
        }
    }
};

// The rows of RowWalk's walk of (px, py, pz), fetched by the 32 lanes of a
// warp at once: row r of the (y, z) box (z-major, the walk's order) goes to
// lane r % 32 of batch r / 32, which applies the walk's pruning and loads
// the row's slot bounds (a pruned row gets an empty range).  row(k) then
// hands every lane the bounds of row k of the current batch.  Every lane of
// the warp must take part (the query point is the same for all).
struct WarpRows {
    const GridDesc& g;
    const WalkBounds& wb;
    const unsigned* __restrict__ start;
    float px, py, pz;
    int z0, y0, ny, nrows;
    unsigned s0, s1;  // this lane's row of the current batch

    __device__ __forceinline__ WarpRows(const GridDesc& g_, const WalkBounds& w_, const unsigned* __restrict__ st,
                                        float x_, float y_, float z_)
        : g(g_), wb(w_), start(st), px(x_), py(y_), pz(z_)
    {
        bool cl = false;
        z0 = cell_coord(pz - wb.reach, g.minf[2], g.inv_d, g.dim[2], &cl);
        const int z1 = cell_coord(pz + wb.reach, g.minf[2], g.inv_d, g.dim[2], &cl);
        y0 = cell_coord(py - wb.reach, g.minf[1], g.inv_d, g.dim[1], &cl);
        const int y1 = cell_coord(py + wb.reach, g.minf[1], g.inv_d, g.dim[1], &cl);
        ny = y1 - y0 + 1;
        nrows = ny * (z1 - z0 + 1);
    }

    // Load batch b (rows 32 b .. 32 b + 31); returns the rows in it.
    __device__ __forceinline__ int batch(int b)
    {
        const int r = 32 * b + (int)(threadIdx.x & 31);
        s0 = s1 = 0;
        if (r < nrows) {
            const int z = z0 + r / ny, yy = y0 + r % ny;
            const float rz = wb.reach2 - axis_gap2(pz, z, g.dim[2], g.minf[2], wb);
            const float ryz = rz - axis_gap2(py, yy, g.dim[1], g.minf[1], wb);
            if (rz > 0.0f && ryz > 0.0f) {
                const float xr = fmaf(ryz, rsqrtf(ryz), wb.margin);
                bool cl = false;
                const int x0 = cell_coord(px - xr, g.minf[0], g.inv_dx, g.dim[0], &cl);
                const int x1 = cell_coord(px + xr, g.minf[0], g.inv_dx, g.dim[0], &cl);
                const unsigned rowk = (unsigned)g.dim[0] * ((unsigned)yy + (unsigned)g.dim[1] * (unsigned)z);
                s0 = __ldg(start + rowk + x0);
                s1 = __ldg(start + rowk + x1 + 1);
            }
        }
        const int left = nrows - 32 * b;
        return left < 32 ? left : 32;
    }

    __device__ __forceinline__ void row(int k, unsigned& r0, unsigned& r1) const
    {
        r0 = __shfl_sync(0xffffffffu, s0, k);
        r1 = __shfl_sync(0xffffffffu, s1, k);
    }

    // After batch(): number the batch's candidates 0 .. total-1 in walk order
    // (rows in order, slots ascending) so that the lanes can take them by
    // flat index.  Returns total.
    unsigned pre;  // this lane's row: first flat index
    __device__ __forceinline__ unsigned flatten()
    {
        const unsigned lane = threadIdx.x & 31;
        const unsigned len = s1 - s0;
        unsigned inc = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned u = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= (unsigned)o) inc += u;
        }
        pre = inc - len;
        return __shfl_sync(0xffffffffu, inc, 31);
    }

    // Slot of flat index k (k < total), for every lane (each its own k).
    __device__ __forceinline__ unsigned slot(unsigned k) const
    {
        int lo = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {  // the last row whose first index <= k
            const unsigned p = __shfl_sync(0xffffffffu, pre, lo + step);
            if (p <= k) lo += step;
        }
        return __shfl_sync(0xffffffffu, s0, lo) + (k - __shfl_sync(0xffffffffu, pre, lo));
    }
};

// ---------------------------------------------------------------- launchers

// One-time kernel attributes; call before any stream capture.
cudaError_t prepare_kernels();

// Exclusive scan of n counts into start[0..n] (start[n] = total).  part must
// hold scan_parts(n) + 1 entries.
int scan_parts(int n);
cudaError_t launch_scan(const unsigned* counts, int n, unsigned* part, unsigned* start,
                        cudaStream_t s, long long* launches);

// The uniform grid over [mn, mx] with cells of size dx along x and d along
// y and z (dim = ceil((mx - mn) / size) per axis, inv = fl(1 / size));
// SPH_ERR_OVERFLOW beyond 2^31 - 2 cells.  make_grid: dx = d.
int make_grid_x(const float mn[3], const float mx[3], float dx, float d, GridDesc* g);
inline int make_grid(const float mn[3], const float mx[3], float d, GridDesc* g)
{
    return make_grid_x(mn, mx, d, d, g);
}

// Cell keys of one grid (the allocation-free binning); err gets
// SPH_DEV_CLAMPED for a position outside [box_min, box_max] or NaN.
cudaError_t launch_keys(const float4* pos, int n, const GridDesc& g, const float box_min[3], const float box_max[3],
                        unsigned* key, unsigned* rank, unsigned* count, unsigned* err, cudaStream_t s,
                        long long* launches);
// Cell keys of every scene's particles (global keys c_base + local key).
cudaError_t launch_scene_keys(const float4* pos, const Scenes& sc, unsigned* key, unsigned* rank,
                              unsigned* count, unsigned* err, cudaStream_t s, long long* launches);
cudaError_t launch_scatter(const unsigned* key, const unsigned* rank, const unsigned* start, int n,
                           int* tmp, cudaStream_t s, long long* launches);
// The same, also tmp_id[dst] = id of the particle (pos.w).
cudaError_t launch_scatter_ids(const unsigned* key, const unsigned* rank, const unsigned* start, const float4* pos,
                               int n, int* tmp, int* tmp_id, cudaStream_t s, long long* launches);
// Per-cell sort by particle id + gather.  big_list (ncells ints) and
// big_count (one u32) are scratch for the cells too large for one warp.
cudaError_t launch_cellsort_gather(const unsigned* start, int ncells, const int* tmp,
                                   const float4* pos_in, const float4* vel_in, float4* pos_out,
                                   float4* vel_out, int nb, int* slot_of_boid, int* big_list,
                                   unsigned* big_count, cudaStream_t s, long long* launches);
// The same with one thread per sorted slot (for grids of small cells); key
// holds the cell of every storage slot, n the number of particles.
// tmp_id: the ids beside tmp (launch_scatter_ids); soa: the SoA copy of
// pos_out (soa_stride(n) floats per axis), written as well.
cudaError_t launch_cellsort_slots(const unsigned* start, const unsigned* key, int n, int ncells,
                                  const int* tmp, const int* tmp_id, const float4* pos_in, const float4* vel_in,
                                  float4* pos_out, float4* vel_out, float* soa, int nb, int* slot_of_boid,
                                  int* big_list, unsigned* big_count, cudaStream_t s, long long* launches);
cudaError_t launch_slot_keys(const unsigned* start, int ncells, unsigned* slot_key, cudaStream_t s,
                             long long* launches);

// Hit segments the density pass keeps per fluid particle for the force
// pass: at most SEG_CAP (first slot, 32-bit pair mask) entries each.
constexpr int SEG_CAP = 128;

// Multiprocessors of the current device (queried once per device).
int sm_count();

// The sorted positions once more as three float arrays (x, y, z of slot j
// at x[j], y[j], z[j]; 8-byte aligned, so slots 2k, 2k + 1 load as one
// float2 per axis): the candidate tests of the neighbour passes read two
// candidates per load and test them with packed float32x2 arithmetic.
struct SoaPos {
    const float* __restrict__ x;
    const float* __restrict__ y;
    const float* __restrict__ z;
};
// Elements per axis of the SoA copy of n positions (even).
__host__ __device__ inline size_t soa_stride(size_t n) { return (n + 1) & ~(size_t)1; }

// Launch shape of the neighbour passes (chosen by the autotuner; results do
// not depend on it).
struct Tuning {
    int block;       // threads per block of density / forces (64 .. 512)
    int use_seg;     // 1: the density pass records hit segments and the force pass reads them
    int pipe_tile;   // > 0: both neighbour passes in one cooperative launch, tiles of this many slots
    int pipe_block;  // threads per block of that launch (128 or 256)
    int ppt;         // particles per thread of the separate neighbour-pass launches (1, 2 or 4)
};

// Density, neighbour counts, candidates tested (ncand) and, with seg given
// and t.use_seg, the hit segments of every fluid particle (seg: SEG_CAP
// entries per particle, nseg: their number).  list (may be NULL = every
// particle) restricts the pass to the sorted slots list[0 .. *list_len)
// (device memory, built on the device); no segments are written then.
// prec (may be NULL): the force pass's 32-byte record of every particle,
// (x, y, z, p) and (v, m / rho with the sign bit set for attached
// particles), read by launch_forces' fluid particles.
cudaError_t launch_density(const float4* pos, const float4* vel, const SoaPos& xyz, const unsigned* start,
                           const Scenes& sc, const Tuning& t, float* rho, float2* ab, float4* prec, int* nbr,
                           uint2* seg, int* nseg, int* ncand, const int* list, const unsigned* list_len,
                           unsigned* err, cudaStream_t s, long long* launches);
// The step's force pass: F_b of every boid (bmask NULL) or of the boids with
// bmask[b] != 0 (their fb.w = 1), a warp per boid, also stored to acc at the
// attached slot when acc is given; with fluid = true also every fluid
// particle, integrated into pos_next/vel_next with the next keys emitted,
// its pairs taken from the density pass's hit segments when t.use_seg (the
// same step's density pass must have written them).  acc, touched, infl:
// the diagnostic fields, written when given (all three or none; attached
// particles get touched = 0, influence = 0).  boids: the F_b warps of the
// boids (bmask NULL = all) take part; fluid: the fluid blocks (pair forces,
// integration, next keys) take part.  One launch.
cudaError_t launch_forces(const float4* pos, const SoaPos& xyz, const float4* vel, const float* rho, const float2* ab,
                          const float4* prec, const unsigned* start, const uint2* seg, const int* nseg,
                          const Scenes& sc,
                          const Tuning& t, const unsigned* list, const unsigned* list_off, size_t list_cap,
                          bool boids, bool fluid, const int* slot_of_boid, const int* bmask, float4* fb,
                          float4* acc, int* touched, float4* infl, float4* pos_next, float4* vel_next,
                          unsigned* key, unsigned* rank, unsigned* count, unsigned* err, cudaStream_t s,
                          long long* launches);
// Both neighbour passes in one cooperative launch (t.pipe_tile > 0):
// density over tiles of sorted slots, a bounded grid barrier
// (SPH_DEV_TIMEOUT if it gives up), then F_b of the boids and the force
// pass; bit for bit launch_density + launch_forces.  queue: 3 device words.
// skip_cta >= 0: test hook, that CTA does not arrive at the barrier.
cudaError_t launch_nbr_pipeline(const float4* pos, const SoaPos& xyz, const float4* vel, const unsigned* start,
                                const Scenes& sc, const Tuning& t, float* rho, float2* ab, float4* prec, int* nbr,
                                uint2* seg, int* nseg, int* ncand, const int* slot_of_boid, float4* fb,
                                float4* acc, int* touched, float4* infl, float4* pos_next, float4* vel_next,
                                unsigned* key, unsigned* rank, unsigned* count, unsigned* queue, int skip_cta,
                                unsigned* err, cudaStream_t s, long long* launches);
// Neighbour lists of every particle at off[i] (exclusive scan of the
// density pass's counts), in walk order; lists ending beyond cap are
// skipped and flagged SPH_DEV_LIST_OVERFLOW.
cudaError_t launch_fill_lists(const float4* pos, const unsigned* start, const Scenes& sc, const unsigned* off,
                              unsigned* list, size_t cap, unsigned* err, cudaStream_t s, long long* launches);
// The lossy fixed-capacity hash grid (ablation): neighbour counts per slot
// through buckets of cap entries per cell; *dropped = entries lost.
// tracker: ncells counters; buckets: ncells * cap entries.
cudaError_t launch_bucket_neighbors(const float4* pos, const unsigned* start, const Scenes& sc, unsigned* tracker,
                                    int ncells, unsigned* buckets, int cap, int* counts, unsigned long long* dropped,
                                    cudaStream_t s, long long* launches);
cudaError_t launch_neighbor_list(const float4* pos, const unsigned* start, const Scenes& sc, int* counts,
                                 const long long* offsets, int* list, cudaStream_t s, long long* launches);

cudaError_t launch_boid_keys(const float4* bpos, const Scenes& sc, unsigned* bkey, unsigned* brank,
                             unsigned* bcount, cudaStream_t s, long long* launches);
// The obstacle grid over the boid grid's cells (one scene): mean outward
// normal and count of the obstacles whose surface passes within half a
// cell diagonal of each cell's centre.  shapes: n_sphere x (centre, radius)
// then n_box x (min, max) floats, device memory.
cudaError_t launch_obstacle_grid(const StepConst& c, const float* shapes, int n_sphere, int n_box, float half_diag,
                                 float4* grid, cudaStream_t s, long long* launches);
// vel_s: the particles' sorted velocities of the step (the attached
// particles' own velocities, read by the literal coupling).
cudaError_t launch_boid_rules(const float4* bpos_s, const float4* bvel_s, const unsigned* bstart,
                              const float4* obst, const Scenes& sc, const float4* fb, const float4* vel_s,
                              float4* bpos, float4* bvel,
                              float4* pos_next, float4* vel_next, const int* slot_of_boid,
                              unsigned* key, unsigned* rank, unsigned* count, unsigned* err,
                              cudaStream_t s, long long* launches);

// Surrogate inputs and outputs (sph_features.cu).  The feature grid pass
// (every fluid particle into the integer sums of its feature cell; grid:
// nfcells int4, zeroed here) and the features of every boid (a warp each).
cudaError_t launch_features(const float4* pos, const float4* vel, const unsigned* start, const float4* bpos,
                            const float4* bvel, const Scenes& sc, int4* grid, int nfcells, void* x, cudaStream_t s,
                            long long* launches);
cudaError_t launch_mark_needed(const float4* pos, const unsigned* start, const Scenes& sc, const int* slot_of_boid,
                               const int* bmask, unsigned char* need, cudaStream_t s, long long* launches);
// list[0 .. *len) = the slots with need[slot] != 0 (order unspecified); *len
// is reset first.
cudaError_t launch_compact_needed(const unsigned char* need, int n, int* list, unsigned* len, cudaStream_t s,
                                  long long* launches);
cudaError_t launch_surrogate_out(const float* y, const void* x, const float* lo, const float* hi, int nb,
                                 float f_scale, float log_err_max, float4* out, int* flag, unsigned* nflag,
                                 cudaStream_t s, long long* launches);

// Surface reconstruction (sph_surface.cu): the voxel density on a grid of
// corners and marching cubes into a triangle buffer.
struct VoxelConst {
    int dims[3];        // corners per axis
    float origin[3];    // corner (0, 0, 0)
    float spacing;
    float R, R2, invR2; // neighbourhood radius, fl(R R), fl(1 / R2)
    float r;            // particle radius
    WalkBounds wb;      // walk bounds of radius R on the particle grid
};
cudaError_t launch_voxel_density(const float4* pos, const unsigned* start, const Scenes& sc, const VoxelConst& v,
                                 float* phi, int* count, cudaStream_t s, long long* launches);
// Host copies of the generated marching-cubes tables (edge: 256 masks, tri:
// 256 x 16, -1 terminated); -1 if the generator failed its own checks.
int mc_tables_host(unsigned short* edge, signed char* tri);
// Copy the tables to the current device's constant memory (once per device).
cudaError_t mc_upload_tables();
// Tiles of consecutive cubes: per-tile counts (each cube's case byte kept
// in cases[ncubes]), one scan of the tile totals, then the triangles from
// each tile's offset (three launches).  tile_count and tile_off hold
// mc_tiles(ncubes) words; *total receives the triangle count.
long long mc_tiles(long long ncubes);
cudaError_t launch_marching_cubes(const float* phi, const int dims[3], const float origin[3], float spacing,
                                  float iso, unsigned char* cases, unsigned* tile_count,
                                  unsigned long long* tile_off, unsigned* total, float* tris,
                                  unsigned long long cap, cudaStream_t s, long long* launches);

// Per-scene step statistics (sph_stats): blocks of STATS_CHUNK slots write
// STATS_PART float64 partials each (part: S x chunks x STATS_PART), one block
// per scene reduces them to STATS_OUT values in out (S x STATS_OUT).
constexpr int STATS_CHUNK = 2048;
constexpr int STATS_PART = 12;
constexpr int STATS_OUT = 12;  // SPH_STATS_N
cudaError_t launch_stats(const float4* pos, const float4* vel, const float* rho, const int* nbr,
                         const unsigned* cell_start, const Scenes& sc, int chunks, double* part, double* out,
                         cudaStream_t s, long long* launches);

// Set the message that sph_last_error(NULL) returns on this thread.
void set_handleless_error(const char* msg);

}  // namespace sphk
