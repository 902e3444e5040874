// sph_physics.cu -- the neighbour passes of the step on the sorted state:
// poly6 density (+ neighbour counts), pressure + viscosity pair forces with
// touched_by_boid / boid_influence, the fluid force on each boid, and the
// Euler-Cromer integration with damped walls fused into the force pass.
//
// Paper: section "Smoothed Particle Hydrodynamics" (poly6 kernel), section
// "Pressure and Viscosity" (equation of state p = k (rho - rho0), the
// symmetrised pressure force with the spiky gradient, the velocity-difference
// viscosity force, their combined pair form), listing "Compute acceleration"
// (touched_by_boid, boid_influence), the frame loop of section "Governing
// Equations" (density -> forces -> integration) and section "Background"
// (damped boundary).
//
// One thread per particle in sorted order.  A thread walks its 27-cell
// stencil as 9 x-rows (cells x-1..x+1 of a row are contiguous in the sorted
// arrays), rows in (dz, dy) order, so its float32 sums have a fixed order
// that depends only on the state.  Neighbouring threads share cells, so the
// candidate loads are served by L1.
#include "sph_internal.cuh"

namespace sphk {

struct RowRange {
    unsigned s0, s1;
};

// The sorted-slot range of the x-row (cx-1 .. cx+1, y, z), clipped to the grid.
__device__ __forceinline__ RowRange row_range(const GridDesc& g, const unsigned* __restrict__ start,
                                              int cx, int y, int z)
{
    int x0 = cx > 0 ? cx - 1 : 0;
    int x1 = cx + 1 < g.dim[0] ? cx + 1 : g.dim[0] - 1;
    unsigned row = (unsigned)g.dim[0] * ((unsigned)y + (unsigned)g.dim[1] * (unsigned)z);
    RowRange r;
    r.s0 = __ldg(start + row + x0);
    r.s1 = __ldg(start + row + x1 + 1);
    return r;
}

// ---------------------------------------------------------------- density

__global__ void __launch_bounds__(256)
k_density(const float4* __restrict__ pos, const unsigned* __restrict__ start, StepConst c,
          float* __restrict__ rho, int* __restrict__ nbr, unsigned* __restrict__ err)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= c.n) return;
    const float4 pi = pos[i];
    const bool att_i = id_of(pi) < c.nb;
    bool clamped = false;
    const int cx = cell_coord(pi.x, c.g.minf[0], c.g.inv_d, c.g.dim[0], &clamped);
    const int cy = cell_coord(pi.y, c.g.minf[1], c.g.inv_d, c.g.dim[1], &clamped);
    const int cz = cell_coord(pi.z, c.g.minf[2], c.g.inv_d, c.g.dim[2], &clamped);
    float sum = 0.0f;
    int cnt = 0;
    for (int dz = -1; dz <= 1; ++dz) {
        int z = cz + dz;
        if (z < 0 || z >= c.g.dim[2]) continue;
        for (int dy = -1; dy <= 1; ++dy) {
            int y = cy + dy;
            if (y < 0 || y >= c.g.dim[1]) continue;
            RowRange rr = row_range(c.g, start, cx, y, z);
            for (unsigned j = rr.s0; j < rr.s1; ++j) {
                const float4 pj = __ldg(pos + j);
                float r2 = pair_r2(__fsub_rn(pj.x, pi.x), __fsub_rn(pj.y, pi.y), __fsub_rn(pj.z, pi.z));
                if (r2 < c.h2) {
                    bool skip = att_i && id_of(pj) < c.nb && j != (unsigned)i;
                    if (!skip) {
                        float t = c.h2 - r2;
                        sum = fmaf(t * t, t, sum);
                        cnt += j != (unsigned)i;
                    }
                }
            }
        }
    }
    float r = c.mC6 * sum;
    rho[i] = r;
    nbr[i] = cnt;
    if (!isfinite(r)) atomicOr(err, SPH_DEV_NONFINITE);
}

cudaError_t launch_density(const float4* pos, const unsigned* start, const StepConst& c, float* rho,
                           int* nbr, unsigned* err, cudaStream_t s, long long* launches)
{
    if (c.n <= 0) return cudaSuccess;
    k_density<<<(c.n + 255) / 256, 256, 0, s>>>(pos, start, c, rho, nbr, err);
    ++*launches;
    return cudaGetLastError();
}

// ------------------------------------------------------- forces + integrate

// f_ij = m/rho_j [ C_p (p_i + p_j)/2 (1-q)^2/q r_ij - C_v mu (1-q) v_ij ],
// r_ij = x_i - x_j, v_ij = v_i - v_j; a_i = (1/rho_i) sum_j f_ij (+ g).
template <int MODE>
__global__ void __launch_bounds__(256)
k_forces(const float4* __restrict__ pos, const float4* __restrict__ vel, const float* __restrict__ rho,
         const unsigned* __restrict__ start, StepConst c, float4* __restrict__ acc,
         int* __restrict__ touched, float4* __restrict__ infl, float4* __restrict__ fb,
         float4* __restrict__ pos_next, float4* __restrict__ vel_next, unsigned* __restrict__ key,
         unsigned* __restrict__ rank, unsigned* __restrict__ count, unsigned* __restrict__ err)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = i < c.n;
    const int ii = active ? i : 0;
    const float4 pi = pos[ii];
    const int id_i = id_of(pi);
    const bool att_i = id_i < c.nb;
    // MODE 1 computes only the attached particles (threads of the others idle)
    const bool work = active && (MODE == 0 || att_i);

    float ax = 0.f, ay = 0.f, az = 0.f;
    float bx = 0.f, by = 0.f, bz = 0.f;
    int touch = 0;
    float rho_i = 1.0f;
    bool clamped = false;
    if (work) {
        const float4 vi = __ldg(vel + i);
        rho_i = __ldg(rho + i);
        const float p_i = c.k * (rho_i - c.rho0);
        const int cx = cell_coord(pi.x, c.g.minf[0], c.g.inv_d, c.g.dim[0], &clamped);
        const int cy = cell_coord(pi.y, c.g.minf[1], c.g.inv_d, c.g.dim[1], &clamped);
        const int cz = cell_coord(pi.z, c.g.minf[2], c.g.inv_d, c.g.dim[2], &clamped);
        for (int dz = -1; dz <= 1; ++dz) {
            int z = cz + dz;
            if (z < 0 || z >= c.g.dim[2]) continue;
            for (int dy = -1; dy <= 1; ++dy) {
                int y = cy + dy;
                if (y < 0 || y >= c.g.dim[1]) continue;
                RowRange rr = row_range(c.g, start, cx, y, z);
                for (unsigned j = rr.s0; j < rr.s1; ++j) {
                    const float4 pj = __ldg(pos + j);
                    const float dx = __fsub_rn(pj.x, pi.x);
                    const float dy_ = __fsub_rn(pj.y, pi.y);
                    const float dz_ = __fsub_rn(pj.z, pi.z);
                    const float r2 = pair_r2(dx, dy_, dz_);
                    if (!(r2 < c.h2) || r2 == 0.0f) continue;
                    const bool att_j = id_of(pj) < c.nb;
                    if (att_i && att_j) continue;
                    const float4 vj = __ldg(vel + j);
                    const float rho_j = __ldg(rho + j);
                    const float p_j = c.k * (rho_j - c.rho0);
                    const float rinv = rsqrtf(r2);
                    const float q = r2 * rinv * c.inv_h;
                    const float omq = 1.0f - q;
                    const float m_rho_j = c.mass / rho_j;
                    // pressure: C_p (p_i+p_j)/2 (1-q)^2 / q along r_ij = -(dx,dy,dz)
                    const float sp = -m_rho_j * c.half_cp_h * (p_i + p_j) * omq * omq * rinv;
                    // viscosity: -C_v mu (1-q) (v_i - v_j)
                    const float sv = -m_rho_j * c.cv_mu * omq;
                    const float fx = fmaf(sp, dx, sv * (vi.x - vj.x));
                    const float fy = fmaf(sp, dy_, sv * (vi.y - vj.y));
                    const float fz = fmaf(sp, dz_, sv * (vi.z - vj.z));
                    ax += fx;
                    ay += fy;
                    az += fz;
                    if (MODE == 0 && att_j) {
                        ++touch;
                        bx += fx;
                        by += fy;
                        bz += fz;
                    }
                }
            }
        }
    }
    const float inv_rho = 1.0f / rho_i;
    ax *= inv_rho;
    ay *= inv_rho;
    az *= inv_rho;

    if (MODE == 1) {
        if (work) fb[id_i] = make_float4(ax, ay, az, 0.0f);
        return;
    }

    // ---- MODE 0: record, integrate, emit the next step's keys
    bool fluid = active && !att_i;
    unsigned k_next = 0;
    if (active) {
        if (att_i) {
            fb[id_i] = make_float4(ax, ay, az, 0.0f);
            acc[i] = make_float4(ax, ay, az, 0.0f);
        } else {
            ax += c.grav[0];
            ay += c.grav[1];
            az += c.grav[2];
            acc[i] = make_float4(ax, ay, az, 0.0f);
        }
        touched[i] = touch;
        infl[i] = make_float4(bx * inv_rho, by * inv_rho, bz * inv_rho, 0.0f);
    }
    if (fluid) {
        const float4 vi = __ldg(vel + i);
        float v[3] = {fmaf(ax, c.dt, vi.x), fmaf(ay, c.dt, vi.y), fmaf(az, c.dt, vi.z)};
        float x[3] = {fmaf(v[0], c.dt, pi.x), fmaf(v[1], c.dt, pi.y), fmaf(v[2], c.dt, pi.z)};
        if (!(isfinite(x[0]) && isfinite(x[1]) && isfinite(x[2]) && isfinite(v[0]) &&
              isfinite(v[1]) && isfinite(v[2])))
            atomicOr(err, SPH_DEV_NONFINITE);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float lo = c.box_min[a], hi = c.box_max[a];
            if (x[a] < lo) {
                x[a] = 2.0f * lo - x[a];
                v[a] = -c.restitution * v[a];
            } else if (x[a] > hi) {
                x[a] = 2.0f * hi - x[a];
                v[a] = -c.restitution * v[a];
            }
            x[a] = fminf(fmaxf(x[a], lo), hi);
        }
        pos_next[i] = make_float4(x[0], x[1], x[2], pi.w);
        vel_next[i] = make_float4(v[0], v[1], v[2], 0.0f);
        k_next = cell_key(c.g, x[0], x[1], x[2], &clamped);
        key[i] = k_next;
    }
    unsigned r = agg_increment(count, k_next, fluid);
    if (fluid) rank[i] = r;
    if (__any_sync(FULL, clamped) && (threadIdx.x & 31) == 0) atomicOr(err, SPH_DEV_CLAMPED);
}

cudaError_t launch_forces(int mode, const float4* pos, const float4* vel, const float* rho,
                          const unsigned* start, const StepConst& c, float4* acc, int* touched,
                          float4* infl, float4* fb, float4* pos_next, float4* vel_next,
                          unsigned* key, unsigned* rank, unsigned* count, unsigned* err,
                          cudaStream_t s, long long* launches)
{
    if (c.n <= 0) return cudaSuccess;
    int blocks = (c.n + 255) / 256;
    if (mode == 0)
        k_forces<0><<<blocks, 256, 0, s>>>(pos, vel, rho, start, c, acc, touched, infl, fb, pos_next,
                                           vel_next, key, rank, count, err);
    else
        k_forces<1><<<blocks, 256, 0, s>>>(pos, vel, rho, start, c, acc, touched, infl, fb, pos_next,
                                           vel_next, key, rank, count, err);
    ++*launches;
    return cudaGetLastError();
}

// ---------------------------------------------------------- neighbour list

__global__ void __launch_bounds__(256)
k_neighbor_list(const float4* __restrict__ pos, const unsigned* __restrict__ start, StepConst c,
                int* __restrict__ counts, const long long* __restrict__ offsets, int* __restrict__ list)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= c.n) return;
    const float4 pi = pos[i];
    const int id_i = id_of(pi);
    const bool att_i = id_i < c.nb;
    bool clamped = false;
    const int cx = cell_coord(pi.x, c.g.minf[0], c.g.inv_d, c.g.dim[0], &clamped);
    const int cy = cell_coord(pi.y, c.g.minf[1], c.g.inv_d, c.g.dim[1], &clamped);
    const int cz = cell_coord(pi.z, c.g.minf[2], c.g.inv_d, c.g.dim[2], &clamped);
    long long o = offsets ? offsets[id_i] : 0;
    int cnt = 0;
    for (int dz = -1; dz <= 1; ++dz) {
        int z = cz + dz;
        if (z < 0 || z >= c.g.dim[2]) continue;
        for (int dy = -1; dy <= 1; ++dy) {
            int y = cy + dy;
            if (y < 0 || y >= c.g.dim[1]) continue;
            RowRange rr = row_range(c.g, start, cx, y, z);
            for (unsigned j = rr.s0; j < rr.s1; ++j) {
                if (j == (unsigned)i) continue;
                const float4 pj = pos[j];
                if (att_i && id_of(pj) < c.nb) continue;
                float r2 = pair_r2(__fsub_rn(pj.x, pi.x), __fsub_rn(pj.y, pi.y), __fsub_rn(pj.z, pi.z));
                if (r2 < c.h2) {
                    if (list) list[o + cnt] = id_of(pj);
                    ++cnt;
                }
            }
        }
    }
    counts[id_i] = cnt;
}

cudaError_t launch_neighbor_list(const float4* pos, const unsigned* start, const StepConst& c,
                                 int* counts, const long long* offsets, int* list, cudaStream_t s,
                                 long long* launches)
{
    if (c.n <= 0) return cudaSuccess;
    k_neighbor_list<<<(c.n + 255) / 256, 256, 0, s>>>(pos, start, c, counts, offsets, list);
    ++*launches;
    return cudaGetLastError();
}

}  // namespace sphk
