// sph_internal.cuh -- device helpers, per-step constants and the handle of the
// GB300 SPH-with-boids step library.  Everything here is internal; the public
// surface is include/sph.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sph.h"

namespace sphk {

constexpr unsigned FULL = 0xffffffffu;

// A uniform grid over the box (section "Neighborhood Search"): dim cells per
// axis, float32 origin and reciprocal cell size used by get_cell.
struct GridDesc {
    int dim[3];
    int ncells;
    float minf[3];
    float inv_d;
};

// Everything a kernel of the step needs, precomputed on the host.
struct StepConst {
    GridDesc g;         // particle grid (cell_size)
    GridDesc gb;        // boid grid (boid_cell_size)
    int n;              // particles: attached + fluid
    int nb;             // boids == attached particles (ids < nb)
    float h2;           // fl(h * h): the neighbour predicate bound
    float mC6;          // m * 315 / (64 pi h^9): poly6 prefactor times mass
    float half_cp_h;    // C_p h / 2: pressure pair prefactor (times 1/r)
    float cv_mu;        // C_v mu: viscosity pair prefactor
    float inv_h, mass, k, rho0, dt;
    float grav[3];      // gravity
    float box_min[3], box_max[3];
    float restitution;
    float rs, rs2, rv2; // boid radii (separation) and squared radii
    float w_sep, w_align, w_coh, sph_dt, v_min, v_max, edge_turn;
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
    int cx = cell_coord(x, g.minf[0], g.inv_d, g.dim[0], clamped);
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

// ---------------------------------------------------------------- launchers

// Exclusive scan of n counts into start[0..n] (start[n] = total).  part must
// hold scan_parts(n) + 1 entries.
int scan_parts(int n);
cudaError_t launch_scan(const unsigned* counts, int n, unsigned* part, unsigned* start,
                        cudaStream_t s, long long* launches);

cudaError_t launch_keys(const float4* pos, int n, const GridDesc& g, unsigned* key, unsigned* rank,
                        unsigned* count, unsigned* err, cudaStream_t s, long long* launches);
cudaError_t launch_scatter(const unsigned* key, const unsigned* rank, const unsigned* start, int n,
                           int* tmp, cudaStream_t s, long long* launches);
// Per-cell sort by particle id + gather.  big_list (ncells ints) and
// big_count (one u32) are scratch for the cells too large for one warp.
cudaError_t launch_cellsort_gather(const unsigned* start, int ncells, const int* tmp,
                                   const float4* pos_in, const float4* vel_in, float4* pos_out,
                                   float4* vel_out, int nb, int* slot_of_boid, int* big_list,
                                   unsigned* big_count, cudaStream_t s, long long* launches);
cudaError_t launch_slot_keys(const unsigned* start, int ncells, unsigned* slot_key, cudaStream_t s,
                             long long* launches);

cudaError_t launch_density(const float4* pos, const unsigned* start, const StepConst& c, float* rho,
                           int* nbr, unsigned* err, cudaStream_t s, long long* launches);
// mode 0: full step (every particle; fluid integrated into pos_next/vel_next,
// next keys emitted); mode 1: only the attached particles' F_b.
cudaError_t launch_forces(int mode, const float4* pos, const float4* vel, const float* rho,
                          const unsigned* start, const StepConst& c, float4* acc, int* touched,
                          float4* infl, float4* fb, float4* pos_next, float4* vel_next,
                          unsigned* key, unsigned* rank, unsigned* count, unsigned* err,
                          cudaStream_t s, long long* launches);
cudaError_t launch_neighbor_list(const float4* pos, const unsigned* start, const StepConst& c,
                                 int* counts, const long long* offsets, int* list, cudaStream_t s,
                                 long long* launches);

cudaError_t launch_boid_keys(const float4* bpos, int nb, const GridDesc& gb, unsigned* bkey,
                             unsigned* brank, unsigned* bcount, cudaStream_t s, long long* launches);
cudaError_t launch_boid_rules(const float4* bpos_s, const float4* bvel_s, const unsigned* bstart,
                              const StepConst& c, const float4* fb, float4* bpos, float4* bvel,
                              float4* pos_next, float4* vel_next, const int* slot_of_boid,
                              unsigned* key, unsigned* rank, unsigned* count, unsigned* err,
                              cudaStream_t s, long long* launches);

// Set the message that sph_last_error(NULL) returns on this thread.
void set_handleless_error(const char* msg);

}  // namespace sphk
