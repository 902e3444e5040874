// sph_boids.cu -- the boid half of the step: boid-grid keys and the boid
// rules with the fluid coupling, one warp per boid.
//
// Paper: section "Underwater Agent Behaviors" (Boid Space spatial hash, Boid
// Grid) and section "Boid Motion and Agent Fluid Interaction": separation
// inside protect_range, alignment and cohesion inside visible_range, edge
// avoidance, speed limit, position update, and the fluid -> boid coupling
// through sph_factor.  The boid also moves its attached particle, which
// pushes the fluid in the next step (the paper attaches particles[id] to
// boids[id]).
//
// Every boid reads the start-of-step snapshot (sorted copies), so the result
// does not depend on the order boids are processed in.  Lanes stride over
// the candidates of the boid cells within r_vis (RowWalk) and the warp
// sums with a fixed butterfly, so the float32 result is deterministic.
#include "sph_internal.cuh"

namespace sphk {

__global__ void __launch_bounds__(256)
k_boid_keys(const float4* __restrict__ bpos, Scenes sc, unsigned* __restrict__ bkey,
            unsigned* __restrict__ brank, unsigned* __restrict__ bcount)
{
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    bool active = b < sc.nb_all;
    unsigned k = 0;
    bool clamped = false;
    if (active) {
        const StepConst& c = sc.c[scene_of(sc.bbase, sc.S, (unsigned)b)];
        float4 p = bpos[b];
        k = (unsigned)c.cb_base + cell_key(c.gb, p.x, p.y, p.z, &clamped);
        bkey[b] = k;
    }
    unsigned r = agg_increment(bcount, k, active);
    if (active) brank[b] = r;
}

cudaError_t launch_boid_keys(const float4* bpos, const Scenes& sc, unsigned* bkey, unsigned* brank,
                             unsigned* bcount, cudaStream_t s, long long* launches)
{
    if (sc.nb_all <= 0) return cudaSuccess;
    k_boid_keys<<<(sc.nb_all + 255) / 256, 256, 0, s>>>(bpos, sc, bkey, brank, bcount);
    ++*launches;
    return cudaGetLastError();
}

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

__device__ __forceinline__ int warp_sum_i(int v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

constexpr int BOID_WARPS = 8;

__global__ void __launch_bounds__(BOID_WARPS * 32)
k_boid_rules(const float4* __restrict__ bpos_s, const float4* __restrict__ bvel_s,
             const unsigned* __restrict__ bstart, const float4* __restrict__ obst, Scenes sc,
             const float4* __restrict__ fb, const float4* __restrict__ vel_s,
             float4* __restrict__ bpos, float4* __restrict__ bvel, float4* __restrict__ pos_next,
             float4* __restrict__ vel_next, const int* __restrict__ slot_of_boid,
             unsigned* __restrict__ key, unsigned* __restrict__ rank, unsigned* __restrict__ count,
             unsigned* __restrict__ err)
{
    const int lane = threadIdx.x & 31;
    const int s = blockIdx.x * BOID_WARPS + (threadIdx.x >> 5);
    if (s >= sc.nb_all) return;  // whole warp
    const StepConst& c = sc.c[scene_of(sc.bbase, sc.S, (unsigned)s)];
    const float4 pb = bpos_s[s];
    const float4 vb = bvel_s[s];
    const int b = id_of(pb);
    float cl[3] = {0.f, 0.f, 0.f};  // separation: sum of d (1 - |d|/r_sep), d = p_b - p_j
    float vs[3] = {0.f, 0.f, 0.f};  // alignment: sum of v_j
    float ps[3] = {0.f, 0.f, 0.f};  // cohesion: sum of (p_j - p_b)
    int nv = 0;
    // boid j at pj with velocity vj (vj is used only within r_vis)
    auto take = [&](const float4& pj, const float4& vj) {
        const float dx = __fsub_rn(pj.x, pb.x);
        const float dy_ = __fsub_rn(pj.y, pb.y);
        const float dz_ = __fsub_rn(pj.z, pb.z);
        const float r2 = pair_r2(dx, dy_, dz_);
        if (r2 < c.rs2) {
            float w = 1.0f - sqrtf(r2) / c.rs;
            w = fminf(fmaxf(w, 0.0f), 1.0f);
            cl[0] -= dx * w;
            cl[1] -= dy_ * w;
            cl[2] -= dz_ * w;
        }
        if (r2 < c.rv2) {
            vs[0] += vj.x;
            vs[1] += vj.y;
            vs[2] += vj.z;
            ps[0] += dx;
            ps[1] += dy_;
            ps[2] += dz_;
            ++nv;
        }
    };
    RowWalk walk(c.gb, c.wb, bstart + c.cb_base, pb.x, pb.y, pb.z);
    unsigned s0, s1;
    while (walk.next(s0, s1)) {
        // lane l takes slots s0 + l, s0 + l + 32, ... in that order, two
        // at a time so that both candidates' loads are in flight together
        unsigned j = s0 + lane;
        for (; j + 32 < s1; j += 64) {
            const float4 pa = bpos_s[j], va = bvel_s[j];
            const float4 pc = bpos_s[j + 32], vc = bvel_s[j + 32];
            if (j != (unsigned)s) take(pa, va);
            if (j + 32 != (unsigned)s) take(pc, vc);
        }
        if (j < s1 && j != (unsigned)s) take(bpos_s[j], bvel_s[j]);
    }
    // obstacle avoidance: the obstacle-grid cells whose centre lies within
    // the visual range (the float32 predicate of the boid pairs), their mean
    // normals weighted obst_near within the protection range; the lanes take
    // the cells of the box of obst_reach cells around the boid's own
    float ob[3] = {0.f, 0.f, 0.f};
    int nob = 0;
    if (c.obst_on) {
        bool cl3 = false;
        int lo[3], n3[3];
        const float pp[3] = {pb.x, pb.y, pb.z};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const int cc = cell_coord(pp[a], c.gb.minf[a], c.gb.inv_d, c.gb.dim[a], &cl3);
            lo[a] = max(cc - c.obst_reach, 0);
            n3[a] = min(cc + c.obst_reach, c.gb.dim[a] - 1) - lo[a] + 1;
        }
        const int total = n3[0] * n3[1] * n3[2];
        const float d = c.wb.d;
        for (int k = lane; k < total; k += 32) {
            const int ix = lo[0] + k % n3[0], iy = lo[1] + (k / n3[0]) % n3[1], iz = lo[2] + k / (n3[0] * n3[1]);
            const float4 g = __ldg(obst + c.cb_base + ix + c.gb.dim[0] * (iy + c.gb.dim[1] * iz));
            if (g.w == 0.0f) continue;
            const float cx = __fadd_rn(__fmul_rn((float)ix + 0.5f, d), c.gb.minf[0]);
            const float cy = __fadd_rn(__fmul_rn((float)iy + 0.5f, d), c.gb.minf[1]);
            const float cz = __fadd_rn(__fmul_rn((float)iz + 0.5f, d), c.gb.minf[2]);
            const float r2 = pair_r2(__fsub_rn(cx, pb.x), __fsub_rn(cy, pb.y), __fsub_rn(cz, pb.z));
            if (r2 < c.rv2) {
                const float w = r2 < c.rs2 ? c.obst_near : 1.0f;
                ob[0] = fmaf(w, g.x, ob[0]);
                ob[1] = fmaf(w, g.y, ob[1]);
                ob[2] = fmaf(w, g.z, ob[2]);
                ++nob;
            }
        }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        cl[a] = warp_sum(cl[a]);
        vs[a] = warp_sum(vs[a]);
        ps[a] = warp_sum(ps[a]);
        ob[a] = warp_sum(ob[a]);
    }
    nv = warp_sum_i(nv);
    nob = warp_sum_i(nob);
    if (lane != 0) return;

    float v[3] = {vb.x, vb.y, vb.z};
    const float p[3] = {pb.x, pb.y, pb.z};
    // 1. separation
#pragma unroll
    for (int a = 0; a < 3; ++a) v[a] = fmaf(c.w_sep, cl[a], v[a]);
    if (nv > 0) {
        const float inv_n = 1.0f / (float)nv;
        // 2. alignment towards the mean velocity of the visible boids
#pragma unroll
        for (int a = 0; a < 3; ++a) v[a] = fmaf(c.w_align, vs[a] * inv_n - v[a], v[a]);
        // 3. cohesion towards their mean position
#pragma unroll
        for (int a = 0; a < 3; ++a) v[a] = fmaf(c.w_coh, ps[a] * inv_n, v[a]);
    }
    // 4. fluid -> boid coupling: v += sph_factor dt F_b; literal coupling:
    // the attached particle is integrated like every particle (F_b plus
    // gravity) and v += sph_factor v_att (the paper's velocity update)
    const float4 f = fb[b];
    float vatt[3] = {0.f, 0.f, 0.f};
    if (c.literal) {
        const float4 va = vel_s[slot_of_boid[b]];
        vatt[0] = fmaf(c.dt, f.x + c.grav[0], va.x);
        vatt[1] = fmaf(c.dt, f.y + c.grav[1], va.y);
        vatt[2] = fmaf(c.dt, f.z + c.grav[2], va.z);
#pragma unroll
        for (int a = 0; a < 3; ++a) v[a] = fmaf(c.sph_factor, vatt[a], v[a]);
    } else {
        v[0] = fmaf(c.sph_dt, f.x, v[0]);
        v[1] = fmaf(c.sph_dt, f.y, v[1]);
        v[2] = fmaf(c.sph_dt, f.z, v[2]);
    }
    // 4b. obstacle avoidance: v += w_obst * (weighted mean of the cells' normals)
    if (nob > 0) {
        const float g = c.w_obst / (float)nob;
#pragma unroll
        for (int a = 0; a < 3; ++a) v[a] = fmaf(g, ob[a], v[a]);
    }
    // 5. edge avoidance
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (p[a] < c.box_min[a]) v[a] += c.edge_turn;
        if (p[a] > c.box_max[a]) v[a] -= c.edge_turn;
    }
    // 6. speed limit
    const float sp = sqrtf(fmaf(v[2], v[2], fmaf(v[1], v[1], v[0] * v[0])));
    float scale = 1.0f;
    if (sp > c.v_max) scale = c.v_max / sp;
    else if (sp > 0.0f && sp < c.v_min) scale = c.v_min / sp;
#pragma unroll
    for (int a = 0; a < 3; ++a) v[a] *= scale;
    // 7. position update
    float x[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) x[a] = fmaf(v[a], c.dt, p[a]);
    if (!(isfinite(x[0]) && isfinite(x[1]) && isfinite(x[2]))) atomicOr(err, SPH_DEV_NONFINITE);

    const float4 np = make_float4(x[0], x[1], x[2], pb.w);
    const float4 nvel = make_float4(v[0], v[1], v[2], 0.0f);
    bpos[b] = np;
    bvel[b] = nvel;
    // the attached particle follows the boid into the next step: its
    // position, and its velocity (force coupling) or its own (literal)
    const int slot = slot_of_boid[b];
    pos_next[slot] = np;
    vel_next[slot] = c.literal ? make_float4(vatt[0], vatt[1], vatt[2], 0.0f) : nvel;
    // a boid outside the tank bins its particle into the nearest cell of the
    // grid (no fluid is there); that is the method's state, not an anomaly
    bool cl2 = false;
    const unsigned k = (unsigned)c.c_base + cell_key(c.g, x[0], x[1], x[2], &cl2);
    key[slot] = k;
    rank[slot] = atomicAdd(&count[k], 1u);
}

cudaError_t launch_boid_rules(const float4* bpos_s, const float4* bvel_s, const unsigned* bstart,
                              const float4* obst, const Scenes& sc, const float4* fb, const float4* vel_s,
                              float4* bpos, float4* bvel,
                              float4* pos_next, float4* vel_next, const int* slot_of_boid,
                              unsigned* key, unsigned* rank, unsigned* count, unsigned* err,
                              cudaStream_t s, long long* launches)
{
    if (sc.nb_all <= 0) return cudaSuccess;
    int blocks = (sc.nb_all + BOID_WARPS - 1) / BOID_WARPS;
    k_boid_rules<<<blocks, BOID_WARPS * 32, 0, s>>>(bpos_s, bvel_s, bstart, obst, sc, fb, vel_s, bpos, bvel, pos_next,
                                                    vel_next, slot_of_boid, key, rank, count, err);
    ++*launches;
    return cudaGetLastError();
}

// ------------------------------------------------------------ obstacles

// The obstacle grid (section "Boid Motion and Agent Fluid Interaction": the
// normals of the obstacles' meshes are attributed to the cells of an
// obstacle grid; analytic spheres and boxes stand in for the meshes): a
// thread per boid-grid cell.  An obstacle counts in a cell when its signed
// distance at the cell's centre is within half a cell diagonal (float32, in
// this fixed order); it adds its outward unit normal at the surface point
// nearest the centre (a box from inside: the normal of its nearest face,
// the lowest axis on ties).  The cell keeps their mean and count.
__global__ void __launch_bounds__(256)
k_obstacle_grid(StepConst c, const float* __restrict__ shapes, int n_sphere, int n_box, float half_diag,
                float4* __restrict__ grid)
{
    const int cell = blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= c.gb.ncells) return;
    const int ix = cell % c.gb.dim[0], iy = (cell / c.gb.dim[0]) % c.gb.dim[1],
              iz = cell / (c.gb.dim[0] * c.gb.dim[1]);
    const float d = c.wb.d;
    const float x[3] = {__fadd_rn(__fmul_rn((float)ix + 0.5f, d), c.gb.minf[0]),
                        __fadd_rn(__fmul_rn((float)iy + 0.5f, d), c.gb.minf[1]),
                        __fadd_rn(__fmul_rn((float)iz + 0.5f, d), c.gb.minf[2])};
    float sum[3] = {0.f, 0.f, 0.f};
    int cnt = 0;
    for (int k = 0; k < n_sphere; ++k) {
        const float* S = shapes + 4 * k;
        const float dx = __fsub_rn(x[0], S[0]), dy = __fsub_rn(x[1], S[1]), dz = __fsub_rn(x[2], S[2]);
        const float q2 = pair_r2(dx, dy, dz);
        const float dist = __fsub_rn(sqrtf(q2), S[3]);
        if (!(fabsf(dist) <= half_diag) || !(q2 > 0.0f)) continue;
        const float inv = 1.0f / sqrtf(q2);
        sum[0] += dx * inv;
        sum[1] += dy * inv;
        sum[2] += dz * inv;
        ++cnt;
    }
    for (int k = 0; k < n_box; ++k) {
        const float* B = shapes + 4 * n_sphere + 6 * k;
        float q[3], m[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            q[a] = fmaxf(__fsub_rn(B[a], x[a]), __fsub_rn(x[a], B[3 + a]));
            m[a] = fmaxf(q[a], 0.0f);
        }
        const bool outside = q[0] > 0.0f || q[1] > 0.0f || q[2] > 0.0f;
        const float dist = outside ? sqrtf(pair_r2(m[0], m[1], m[2])) : fmaxf(q[0], fmaxf(q[1], q[2]));
        if (!(fabsf(dist) <= half_diag)) continue;
        float n[3] = {0.f, 0.f, 0.f};
        if (outside) {
#pragma unroll
            for (int a = 0; a < 3; ++a) n[a] = x[a] > B[3 + a] ? m[a] : (x[a] < B[a] ? -m[a] : 0.0f);
            const float inv = 1.0f / dist;
#pragma unroll
            for (int a = 0; a < 3; ++a) n[a] *= inv;
        } else {
            int ax = 0;
            if (q[1] > q[ax]) ax = 1;
            if (q[2] > q[ax]) ax = 2;
            n[ax] = __fsub_rn(x[ax], B[3 + ax]) >= __fsub_rn(B[ax], x[ax]) ? 1.0f : -1.0f;
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) sum[a] += n[a];
        ++cnt;
    }
    const float inv = cnt ? 1.0f / (float)cnt : 0.0f;
    grid[cell] = make_float4(sum[0] * inv, sum[1] * inv, sum[2] * inv, (float)cnt);
}

cudaError_t launch_obstacle_grid(const StepConst& c, const float* shapes, int n_sphere, int n_box, float half_diag,
                                 float4* grid, cudaStream_t s, long long* launches)
{
    if (c.gb.ncells <= 0) return cudaSuccess;
    k_obstacle_grid<<<(c.gb.ncells + 255) / 256, 256, 0, s>>>(c, shapes, n_sphere, n_box, half_diag,
                                                             grid + c.cb_base);
    ++*launches;
    return cudaGetLastError();
}

}  // namespace sphk
