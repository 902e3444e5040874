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
// One thread per particle in sorted order.  A thread walks the cells its
// h-sphere can reach as rows of contiguous sorted slots (RowWalk: rows in
// z, y order, x ascending, each row clipped to the sphere), so its float32
// sums have a fixed order that depends only on the state.  Neighbouring
// threads share cells, so the candidate loads are served by L1.
#include "sph_internal.cuh"

namespace sphk {

// ---------------------------------------------------------------- density

// Hit segments.  The density pass tests every candidate of a fluid
// particle's walk; it also keeps, for the force pass, which candidates are
// within h (r2 < h2: the particle itself and coincident particles among
// them; the force pass skips those by r2 == 0).  Each row of the walk is cut
// into pieces of at most 32 consecutive slots and every piece with a hit is
// stored as one segment (first slot, 32-bit mask of its hits), in walk
// order, at seg[i * SEG_CAP + k]; nseg[i] is the number of segments
// (SEG_CAP + 1 and more: the list did not fit, the force pass tests the
// candidates itself).  The neighbour count is the hits' popcount less one.  The force pass
// then evaluates the pairs in exactly the walk's order without testing a
// candidate again, and the lanes of a warp take their next pair together
// instead of waiting at each row for the lane with the most hits in it.
//
// Besides rho_i it stores ab[i] = (m / rho_i, k (rho_i - rho0)): the two
// per-particle factors of the pair force, so that the force pass divides
// once per particle instead of once per pair (same float32 values).
//
// A fluid particle has no excluded pairs, so its loop counts every hit and
// subtracts the self pair (always visited: r2 = 0) at the end; the sums
// take the same terms in the same order as the attached particles' loop.
template <bool SEG>
__device__ __forceinline__ void density_at(int i, const float4* __restrict__ pos, const float4* __restrict__ vel,
                                           const SoaPos& xyz, const unsigned* __restrict__ start,
                                           const Scenes& sc, float* __restrict__ rho, float2* __restrict__ ab,
                                           float4* __restrict__ prec, int* __restrict__ nbr,
                                           uint2* __restrict__ seg, int* __restrict__ nseg,
                                           int* __restrict__ ncand, unsigned* __restrict__ err)
{
    const StepConst& c = sc.c[scene_of(sc.pbase, sc.S, (unsigned)i)];
    const float h2 = c.h2;
    const int nb_all = sc.nb_all;
    const float4 pi = pos[i];
    const bool att_i = id_of(pi) < nb_all;
    float sum = 0.0f;
    int cnt = 0;
    int nc = 0;
    RowWalk walk(c.g, c.wg, start + c.c_base, pi.x, pi.y, pi.z);
    unsigned s0, s1;
    if (!att_i) {
        // candidates in slot order: an odd first slot alone, then slot
        // pairs (2k, 2k + 1) from the SoA copy, tested side by side with
        // packed float32x2 operations (each component rounded exactly as
        // the scalar form), then an odd last slot alone.  m collects the
        // hits of the current segment (bit = slot - segment start; the
        // particle itself and coincident particles are among them, the force
        // pass skips them by r2 == 0).
        unsigned m = 0;
        auto take = [&](const float4& pj, unsigned sh) {
            const float r2 = pair_r2(__fsub_rn(pj.x, pi.x), __fsub_rn(pj.y, pi.y), __fsub_rn(pj.z, pi.z));
            if (r2 < h2) {
                const float t = h2 - r2;
                sum = fmaf(t * t, t, sum);
                if (SEG) m |= 1u << sh; else ++cnt;
            }
        };
        // x_j - x_i as x_j + (-x_i) and h2 - r2 as fma(r2, -1, h2): the
        // same roundings as the subtractions
        const float2 nx2 = make_float2(-pi.x, -pi.x), ny2 = make_float2(-pi.y, -pi.y), nz2 = make_float2(-pi.z, -pi.z);
        const float2 h22 = make_float2(h2, h2), m11 = make_float2(-1.0f, -1.0f);
        auto take2 = [&](float2 X, float2 Y, float2 Z, unsigned sh) {
            const float2 dx = __fadd2_rn(X, nx2), dy = __fadd2_rn(Y, ny2), dz = __fadd2_rn(Z, nz2);
            const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
            const float2 t = __ffma2_rn(r2, m11, h22);
            const float2 tt = __fmul2_rn(t, t);
            const unsigned bit = SEG ? 1u << sh : 0u;
            if (r2.x < h2) {
                sum = fmaf(tt.x, t.x, sum);
                if (SEG) m |= bit; else ++cnt;
            }
            if (r2.y < h2) {
                sum = fmaf(tt.y, t.y, sum);
                if (SEG) m |= bit << 1; else ++cnt;
            }
        };
        const float2* __restrict__ X2 = reinterpret_cast<const float2*>(xyz.x);
        const float2* __restrict__ Y2 = reinterpret_cast<const float2*>(xyz.y);
        const float2* __restrict__ Z2 = reinterpret_cast<const float2*>(xyz.z);
        // the slots [a, e) with bits relative to b
        auto slots = [&](unsigned a, unsigned e, unsigned b) {
            unsigned j = a;
            if (j & 1u) {
                take(__ldg(pos + j), j - b);
                ++j;
            }
            const unsigned e2 = e & ~1u;
            // two slot pairs (four candidates) in flight per iteration
            for (; j + 4 <= e2; j += 4) {
                const unsigned k = j >> 1;
                const float2 xa = __ldg(X2 + k), ya = __ldg(Y2 + k), za = __ldg(Z2 + k);
                const float2 xb = __ldg(X2 + k + 1), yb = __ldg(Y2 + k + 1), zb = __ldg(Z2 + k + 1);
                take2(xa, ya, za, j - b);
                take2(xb, yb, zb, j + 2 - b);
            }
            if (j < e2) {
                const unsigned k = j >> 1;
                take2(__ldg(X2 + k), __ldg(Y2 + k), __ldg(Z2 + k), j - b);
                j += 2;
            }
            if (j < e) take(__ldg(pos + j), j - b);
        };
        int ns = 0;
        uint2* __restrict__ mine = SEG ? seg + (size_t)i * SEG_CAP : nullptr;
        while (walk.next(s0, s1)) {
            if (!SPH_IN_BOUNDS(s1 - 1u, sc.n_all, err)) break;  // the row's last slot
            nc += (int)(s1 - s0);
            if (SEG) {
                for (unsigned b = s0; b < s1; b += 32u) {
                    m = 0;
                    slots(b, min(b + 32u, s1), b);
                    if (m) {
                        cnt += __popc(m);
                        if (ns < SEG_CAP) mine[ns] = make_uint2(b, m);
                        ++ns;
                    }
                }
            } else {
                slots(s0, s1, s0);
            }
        }
        --cnt;  // the particle itself
        if (SEG) nseg[i] = ns;
    } else {
        while (walk.next(s0, s1)) {
            if (!SPH_IN_BOUNDS(s1 - 1u, sc.n_all, err)) break;
            for (unsigned j = s0; j < s1; ++j) {
                const float4 pj = __ldg(pos + j);
                const float r2 =
                    pair_r2(__fsub_rn(pj.x, pi.x), __fsub_rn(pj.y, pi.y), __fsub_rn(pj.z, pi.z));
                const bool att_pair = id_of(pj) < nb_all;
                if (r2 < h2 && !(att_pair && j != (unsigned)i)) {
                    const float t = h2 - r2;
                    sum = fmaf(t * t, t, sum);
                    cnt += j != (unsigned)i;
                }
            }
            nc += (int)(s1 - s0);
        }
        if (SEG) nseg[i] = 0;  // attached particles are not integrated
    }
    ncand[i] = nc;
    const float r = c.mC6 * sum;
    rho[i] = r;
    const float2 abi = make_float2(c.mass / r, c.k * (r - c.rho0));
    ab[i] = abi;
    if (prec) {  // the force pass's record of j: (x, y, z, p) and (v, m / rho, negative if attached)
        const float4 v = __ldg(vel + i);
        prec[2 * i] = make_float4(pi.x, pi.y, pi.z, abi.y);
        prec[2 * i + 1] = make_float4(v.x, v.y, v.z, att_i ? -abi.x : abi.x);
    }
    nbr[i] = cnt;
    if (!isfinite(r)) atomicOr(err, SPH_DEV_NONFINITE);
}

// Every particle (thread i = slot i).
template <bool SEG>
__global__ void __launch_bounds__(512, 3)
k_density(const float4* __restrict__ pos, const float4* __restrict__ vel, SoaPos xyz,
          const unsigned* __restrict__ start, Scenes sc, float* __restrict__ rho, float2* __restrict__ ab,
          float4* __restrict__ prec, int* __restrict__ nbr, uint2* __restrict__ seg, int* __restrict__ nseg,
          int* __restrict__ ncand, unsigned* __restrict__ err)
{
    // particles t, t + T, t + 2T, ... (T the threads of the grid: a grid of
    // n / ppt threads gives each thread ppt particles)
    const int T = gridDim.x * blockDim.x;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < sc.n_all; t += T)
        density_at<SEG>(t, pos, vel, xyz, start, sc, rho, ab, prec, nbr, seg, nseg, ncand, err);
}


// Only the slots of a list whose length the device holds (the list is built
// on the device; warps stride over it): a warp per particle, the lanes fetch
// the walk's rows together and test a row's candidates side by side, then
// the hits are added in slot order by the same fused multiply-adds as the
// one-thread pass (the lanes pass the terms by shuffles), so the density is
// bit for bit the full pass's.  Kept for few particles (the exact-local
// path), where the one-thread walk leaves its latency exposed.
__global__ void __launch_bounds__(256)
k_density_list(const float4* __restrict__ pos, const unsigned* __restrict__ start, Scenes sc,
               float* __restrict__ rho, float2* __restrict__ ab, int* __restrict__ nbr, int* __restrict__ ncand,
               const int* __restrict__ list, const unsigned* __restrict__ list_len, unsigned* __restrict__ err)
{
    const int lane = threadIdx.x & 31;
    const int nw = gridDim.x * (blockDim.x >> 5);
    const int len = (int)min(*list_len, (unsigned)sc.n_all);
    for (int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w < len; w += nw) {
        const int i = list[w];
        const StepConst& c = sc.c[scene_of(sc.pbase, sc.S, (unsigned)i)];
        const float h2 = c.h2;
        const int nb_all = sc.nb_all;
        const float4 pi = pos[i];
        const bool att_i = id_of(pi) < nb_all;
        float sum = 0.0f;
        int cnt = 0, nc = 0;
        WarpRows rows(c.g, c.wg, start + c.c_base, pi.x, pi.y, pi.z);
        for (int bt = 0; 32 * bt < rows.nrows; ++bt) {
            rows.batch(bt);
            const unsigned total = rows.flatten();
            nc += (int)total;
            for (unsigned k0 = 0; k0 < total; k0 += 32) {
                const unsigned k = k0 + (unsigned)lane;
                const unsigned j = rows.slot(k < total ? k : total - 1);
                bool hit = false, self = false;
                float t = 0.0f;
                if (k < total) {
                    const float4 pj = __ldg(pos + j);
                    const float r2 = pair_r2(__fsub_rn(pj.x, pi.x), __fsub_rn(pj.y, pi.y), __fsub_rn(pj.z, pi.z));
                    self = j == (unsigned)i;
                    hit = r2 < h2 && !(att_i && !self && id_of(pj) < nb_all);
                    t = h2 - r2;
                }
                unsigned m = __ballot_sync(FULL, hit);
                cnt += __popc(m & ~__ballot_sync(FULL, self));
                while (m) {  // the hits in walk order, one fused multiply-add each
                    const int q = __ffs(m) - 1;
                    m &= m - 1u;
                    const float v = __shfl_sync(FULL, t, q);
                    sum = fmaf(v * v, v, sum);
                }
            }
        }
        if (lane == 0) {
            ncand[i] = nc;
            const float r = c.mC6 * sum;
            rho[i] = r;
            ab[i] = make_float2(c.mass / r, c.k * (r - c.rho0));
            nbr[i] = cnt;
            if (!isfinite(r)) atomicOr(err, SPH_DEV_NONFINITE);
        }
    }
}

cudaError_t launch_density(const float4* pos, const float4* vel, const SoaPos& xyz, const unsigned* start,
                           const Scenes& sc, const Tuning& t, float* rho, float2* ab, float4* prec, int* nbr,
                           uint2* seg, int* nseg, int* ncand, const int* list, const unsigned* list_len,
                           unsigned* err, cudaStream_t s, long long* launches)
{
    if (sc.n_all <= 0) return cudaSuccess;
    const int per_block = t.block * (t.ppt > 1 ? t.ppt : 1);
    const int all = (sc.n_all + per_block - 1) / per_block;
    if (list) {
        const int cap = 16 * sm_count();  // 8 warps per block, 16 blocks per SM at most
        const int blocks = (sc.n_all + 7) / 8 < cap ? (sc.n_all + 7) / 8 : cap;
        k_density_list<<<blocks, 256, 0, s>>>(pos, start, sc, rho, ab, nbr, ncand, list, list_len, err);
    } else if (seg && t.use_seg) {
        k_density<true><<<all, t.block, 0, s>>>(pos, vel, xyz, start, sc, rho, ab, prec, nbr, seg, nseg, ncand, err);
    } else {
        k_density<false><<<all, t.block, 0, s>>>(pos, vel, xyz, start, sc, rho, ab, prec, nbr, seg, nseg, ncand,
                                                 err);
    }
    ++*launches;
    return cudaGetLastError();
}

// ------------------------------------------------------- forces + integrate

// f_ij = m/rho_j [ C_p (p_i + p_j)/2 (1-q)^2/q r_ij - C_v mu (1-q) v_ij ],
// r_ij = x_i - x_j, v_ij = v_i - v_j; a_i = (1/rho_i) sum_j f_ij (+ g).
// d = x_j - x_i (float32; x and y packed), r2 its squared norm,
// ab_j = (m / rho_j, p_j).  Every operation is rounded once, in the order
// written (intrinsics, no contraction), and every caller (the force pass,
// the boids' F_b, the list and stream variants) uses this one function,
// so a pair contributes the same bits wherever it is summed.
struct PairTerms {
    float4 pi, vi;
    float p_i, n_hcp, n_cv, inv_h;  // n_hcp = -C_p h / 2, n_cv = -C_v mu

    __device__ __forceinline__ void set(const StepConst& c, const float4& pos_i, const float4& vel_i, float p)
    {
        pi = pos_i;
        vi = vel_i;
        p_i = p;
        n_hcp = -c.half_cp_h;
        n_cv = -c.cv_mu;
        inv_h = c.inv_h;
    }

    __device__ __forceinline__ void add(float2 dxy, float dz, float r2, const float4& vj, float2 abj, float2& fxy,
                                        float& fz) const
    {
        const float rinv = rsqrtf(r2);
        const float omq = __fmaf_rn(-__fmul_rn(r2, rinv), inv_h, 1.0f);  // 1 - q
        const float s = __fmul_rn(abj.x, omq);                          // m/rho_j (1 - q)
        // pressure: -C_p h/2 (p_i + p_j) m/rho_j (1-q)^2 / r along d
        const float sp = __fmul_rn(__fmul_rn(__fmul_rn(__fadd_rn(p_i, abj.y), n_hcp), __fmul_rn(s, omq)), rinv);
        // viscosity: -C_v mu m/rho_j (1-q) (v_i - v_j)
        const float sv = __fmul_rn(s, n_cv);
        const float2 dv = __ffma2_rn(make_float2(vj.x, vj.y), make_float2(-1.0f, -1.0f), make_float2(vi.x, vi.y));
        fxy = __ffma2_rn(make_float2(sp, sp), dxy, __fmul2_rn(make_float2(sv, sv), dv));
        fz = __fmaf_rn(sp, dz, __fmul_rn(sv, __fsub_rn(vi.z, vj.z)));
    }
};

// Loads of what the density pass wrote (densities, (m/rho, p), pair
// records, hit segments): through the read-only path when an earlier launch
// wrote them (COH = false), or as coherent cached loads when the same launch
// wrote them before a grid barrier and an acquire fence (COH = true, the
// fused pipeline; the read-only path is not coherent with such writes).
template <bool COH, class T>
__device__ __forceinline__ T ldd(const T* p)
{
    if constexpr (COH) return __ldca(p);
    else return __ldg(p);
}

// The 32-byte pair record of a particle, (x, y, z, p) and (v, +-m / rho),
// in one 256-bit load (records are 32-byte aligned).
template <bool COH>
__device__ __forceinline__ void ld_rec(const float4* __restrict__ p, float4& a, float4& b)
{
    if constexpr (COH)
        asm volatile("ld.global.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                     : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
                     : "l"(p)
                     : "memory");
    else
        asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
            : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
            : "l"(p));
}

// x_j - x_i, y_j - y_i as one packed addition of (-x_i, -y_i): the same
// roundings as the subtractions.
__device__ __forceinline__ float2 dxy_of(const float4& pj, float2 nxy)
{
    return __fadd2_rn(make_float2(pj.x, pj.y), nxy);
}

// F_b of boid b (section "Boid Motion and Agent Fluid Interaction"): the acceleration
// of its attached particle from the fluid particles within h.  One warp per
// boid: the lanes fetch the walk's rows together (WarpRows) and take its
// candidates by flat index (lane l: candidates l, l + 32, ... in walk
// order), each keeping its own sum, and a butterfly adds the 32 sums (a
// fixed order).
template <bool COH>
__device__ __forceinline__ void boid_fb_warp(int b, int lane, const float4* __restrict__ pos,
                                             const float4* __restrict__ vel, const float* __restrict__ rho,
                                             const float2* __restrict__ ab, const unsigned* __restrict__ start,
                                             const Scenes& sc, const int* __restrict__ slot_of_boid,
                                             const int* __restrict__ bmask, float4* __restrict__ fb,
                                             float4* __restrict__ acc)
{
    const int i = slot_of_boid[b];
    const StepConst& c = sc.c[scene_of(sc.pbase, sc.S, (unsigned)i)];
    const int nb_all = sc.nb_all;
    PairTerms T;
    T.set(c, pos[i], vel[i], ldd<COH>(ab + i).y);
    const float2 nxy = make_float2(-T.pi.x, -T.pi.y);
    const float h2 = c.h2;
    float2 axy = make_float2(0.f, 0.f);
    float az = 0.f;
    WarpRows rows(c.g, c.wg, start + c.c_base, T.pi.x, T.pi.y, T.pi.z);
    for (int bt = 0; 32 * bt < rows.nrows; ++bt) {
        rows.batch(bt);
        const unsigned total = rows.flatten();
        for (unsigned k0 = 0; k0 < total; k0 += 32) {
            const unsigned k = k0 + (unsigned)lane;
            const unsigned j = rows.slot(k < total ? k : total - 1);
            if (k >= total) continue;
            const float4 pj = __ldg(pos + j);
            const float2 dxy = dxy_of(pj, nxy);
            const float dz = __fsub_rn(pj.z, T.pi.z);
            const float r2 = pair_r2(dxy.x, dxy.y, dz);
            if (r2 < h2 && r2 != 0.0f && id_of(pj) >= nb_all) {
                float2 fxy;
                float fz;
                T.add(dxy, dz, r2, __ldg(vel + j), ldd<COH>(ab + j), fxy, fz);
                axy = __fadd2_rn(axy, fxy);
                az = __fadd_rn(az, fz);
            }
        }
    }
    float ax = axy.x, ay = axy.y;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ax += __shfl_xor_sync(FULL, ax, o);
        ay += __shfl_xor_sync(FULL, ay, o);
        az += __shfl_xor_sync(FULL, az, o);
    }
    if (lane == 0) {
        const float inv_rho = 1.0f / ldd<COH>(rho + i);
        const float4 f = make_float4(ax * inv_rho, ay * inv_rho, az * inv_rho, 0.0f);
        fb[b] = make_float4(f.x, f.y, f.z, bmask ? 1.0f : 0.0f);
        if (acc) acc[i] = f;
    }
}

// The arguments of the force pass (k_forces and the fused pipeline).
struct ForceArgs {
    const float4* __restrict__ pos;
    SoaPos xyz;
    const float4* __restrict__ vel;
    const float* rho;
    const float2* ab;
    const float4* prec;
    const unsigned* __restrict__ start;
    const uint2* seg;
    const int* nseg;
    Scenes sc;
    const unsigned* __restrict__ list;
    const unsigned* __restrict__ list_off;
    unsigned list_cap;
    const int* __restrict__ slot_of_boid;
    const int* __restrict__ bmask;
    float4* __restrict__ fb;
    float4* __restrict__ acc;
    int* __restrict__ touched;
    float4* __restrict__ infl;
    float4* __restrict__ pos_next;
    float4* __restrict__ vel_next;
    unsigned* __restrict__ key;
    unsigned* __restrict__ rank;
    unsigned* __restrict__ count;
    unsigned* __restrict__ err;
};

// The force pass of sorted slot i (i >= n_all: an idle lane): pair forces
// with touched_by_boid and boid_influence, gravity, Euler-Cromer
// integration, damped walls and the next step's cell keys.  A fluid
// particle takes its pairs from (in this order of preference) the
// neighbour list, the density pass's hit segments, or a walk that tests the
// candidates again; all three visit the same pairs in the same order.
// acc, touched and infl (the diagnostic fields) are written only when given
// (all three or none); attached particles then record touched = 0 and
// influence = 0 (attached pairs are excluded).  Every lane of the warp
// must call it (warp-aggregated counting).
template <bool COH>
__device__ __forceinline__ void force_particle(const ForceArgs& a, int i)
{
    const float4* __restrict__ pos = a.pos;
    const SoaPos& xyz = a.xyz;
    const float4* __restrict__ vel = a.vel;
    const float* rho = a.rho;
    const float2* ab = a.ab;
    const float4* prec = a.prec;
    const unsigned* __restrict__ start = a.start;
    const uint2* seg = a.seg;
    const int* nseg = a.nseg;
    const Scenes& sc = a.sc;
    const unsigned* __restrict__ list = a.list;
    const unsigned* __restrict__ list_off = a.list_off;
    const unsigned list_cap = a.list_cap;
    float4* __restrict__ acc = a.acc;
    int* __restrict__ touched = a.touched;
    float4* __restrict__ infl = a.infl;
    float4* __restrict__ pos_next = a.pos_next;
    float4* __restrict__ vel_next = a.vel_next;
    unsigned* __restrict__ key = a.key;
    unsigned* __restrict__ rank = a.rank;
    unsigned* __restrict__ count = a.count;
    unsigned* __restrict__ err = a.err;
    const bool active = i < sc.n_all;
    const int ii = active ? i : 0;
    const StepConst& c = sc.c[scene_of(sc.pbase, sc.S, (unsigned)ii)];
    const int nb_all = sc.nb_all;
    const float4 pi = pos[ii];
    const bool fluid = active && id_of(pi) >= nb_all;
    const unsigned* cstart = start + c.c_base;

    float2 axy = make_float2(0.f, 0.f), bxy = make_float2(0.f, 0.f);
    float az = 0.f, bz = 0.f;
    int touch = 0;
    float rho_i = 1.0f;
    bool clamped = false;
    if (fluid) {
        PairTerms T;
        T.set(c, pi, __ldg(vel + i), ldd<COH>(ab + i).y);
        rho_i = ldd<COH>(rho + i);
        const float2 nxy = make_float2(-pi.x, -pi.y);
        // one neighbour j (r2 < h2) from its record (one 32-byte load); the
        // particle itself and coincident particles (r2 = 0) add nothing
        auto pair = [&](unsigned j) {
            if (!SPH_IN_BOUNDS(j, sc.n_all, err)) return;  // a hit segment's slot
            float4 q0, q1;
            ld_rec<COH>(prec + 2 * (size_t)j, q0, q1);
            const float2 dxy = dxy_of(q0, nxy);
            const float dz = __fsub_rn(q0.z, pi.z);
            const float r2 = pair_r2(dxy.x, dxy.y, dz);
            float2 fxy;
            float fz;
            T.add(dxy, dz, r2, q1, make_float2(fabsf(q1.w), q0.w), fxy, fz);
            if (r2 != 0.0f) {
                axy = __fadd2_rn(axy, fxy);
                az = __fadd_rn(az, fz);
                if (__float_as_int(q1.w) < 0) {  // j is attached to a boid
                    ++touch;
                    bxy = __fadd2_rn(bxy, fxy);
                    bz = __fadd_rn(bz, fz);
                }
            }
        };
        unsigned o0 = 0, o1 = 0;
        if (list) {
            o0 = __ldg(list_off + i);
            o1 = __ldg(list_off + i + 1);
        }
        const int ns = seg ? ldd<COH>(nseg + i) : SEG_CAP + 1;
        if (list && o1 <= list_cap) {
            // the neighbour list, in walk order (coincident particles skipped)
            for (unsigned k = o0; k < o1; ++k) {
                const unsigned j = __ldg(list + k);
                const float4 pj = __ldg(pos + j);
                if (pair_r2(__fsub_rn(pj.x, pi.x), __fsub_rn(pj.y, pi.y), __fsub_rn(pj.z, pi.z)) != 0.0f) pair(j);
            }
        } else if (ns <= SEG_CAP) {
            // the density pass's hit segments: one pair per iteration, the
            // next segment fetched while the current pair is evaluated
            const uint2* __restrict__ mine = seg + (size_t)i * SEG_CAP;
            uint2 cur = ns > 0 ? ldd<COH>(mine) : make_uint2(0u, 0u);
            int k = 1;
            while (cur.y) {
                const unsigned j = cur.x + (unsigned)(__ffs(cur.y) - 1);
                cur.y &= cur.y - 1u;
                if (!cur.y && k < ns) cur = ldd<COH>(mine + k++);
                pair(j);
            }
        } else {
            // test a chunk of up to 32 candidates into a bit mask, then run
            // the pair code over the set bits (slot pairs from the SoA copy,
            // as in the density pass)
            const float h2 = c.h2;
            const float2 nx2 = make_float2(-pi.x, -pi.x), ny2 = make_float2(-pi.y, -pi.y),
                         nz2 = make_float2(-pi.z, -pi.z);
            const float2* __restrict__ X2 = reinterpret_cast<const float2*>(xyz.x);
            const float2* __restrict__ Y2 = reinterpret_cast<const float2*>(xyz.y);
            const float2* __restrict__ Z2 = reinterpret_cast<const float2*>(xyz.z);
            auto test1 = [&](unsigned j) {
                const float4 pj = __ldg(pos + j);
                const float r2 = pair_r2(__fsub_rn(pj.x, pi.x), __fsub_rn(pj.y, pi.y), __fsub_rn(pj.z, pi.z));
                return (unsigned)(r2 < h2 && r2 != 0.0f);
            };
            auto test2 = [&](float2 X, float2 Y, float2 Z) {
                const float2 dx = __fadd2_rn(X, nx2), dy = __fadd2_rn(Y, ny2), dz = __fadd2_rn(Z, nz2);
                const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
                return (unsigned)(r2.x < h2 && r2.x != 0.0f) | (unsigned)(r2.y < h2 && r2.y != 0.0f) << 1;
            };
            RowWalk walk(c.g, c.wg, cstart, pi.x, pi.y, pi.z);
            unsigned s0, s1;
            while (walk.next(s0, s1)) {
                for (unsigned base = s0; base < s1; base += 32) {
                    const unsigned e = min(base + 32u, s1);
                    unsigned m = 0, j = base;
                    if (j & 1u) m = test1(j++);
                    const unsigned e2 = e & ~1u;
                    for (; j + 4 <= e2; j += 4) {
                        const unsigned k = j >> 1;
                        const float2 xa = __ldg(X2 + k), ya = __ldg(Y2 + k), za = __ldg(Z2 + k);
                        const float2 xb = __ldg(X2 + k + 1), yb = __ldg(Y2 + k + 1), zb = __ldg(Z2 + k + 1);
                        m |= test2(xa, ya, za) << (j - base);
                        m |= test2(xb, yb, zb) << (j + 2 - base);
                    }
                    if (j < e2) {
                        const unsigned k = j >> 1;
                        m |= test2(__ldg(X2 + k), __ldg(Y2 + k), __ldg(Z2 + k)) << (j - base);
                        j += 2;
                    }
                    if (j < e) m |= test1(j) << (j - base);
                    while (m) {
                        const int t = __ffs(m) - 1;
                        m &= m - 1u;
                        pair(base + (unsigned)t);
                    }
                }
            }
        }
    }
    const float inv_rho = 1.0f / rho_i;
    float ax = axy.x * inv_rho, ay = axy.y * inv_rho;
    az *= inv_rho;
    const float bx = bxy.x, by = bxy.y;

    unsigned k_next = 0;
    if (active && touched) {
        touched[i] = touch;
        infl[i] = make_float4(bx * inv_rho, by * inv_rho, bz * inv_rho, 0.0f);
    }
    if (fluid) {
        ax += c.grav[0];
        ay += c.grav[1];
        az += c.grav[2];
        if (acc) acc[i] = make_float4(ax, ay, az, 0.0f);
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
        bool cl = false;
        k_next = (unsigned)c.c_base + cell_key(c.g, x[0], x[1], x[2], &cl);
        key[i] = k_next;
        clamped = outside_box(c, x[0], x[1], x[2]);  // NaN only: the walls keep x in the box
    }
    unsigned r = agg_increment(count, k_next, fluid);
    if (fluid) rank[i] = r;
    if (__any_sync(FULL, clamped) && (threadIdx.x & 31) == 0) atomicOr(err, SPH_DEV_CLAMPED);
}

// The step's force pass.  The first boid_blocks blocks compute F_b, a warp
// per boid (boid_fb_warp; F_b also goes to acc at the attached slot when
// acc is given); they come first in the grid so that these latency-bound
// warps run alongside the fluid blocks.  The remaining blocks (possibly
// none) take a particle per thread (force_particle).
__global__ void __launch_bounds__(512)
k_forces(ForceArgs a, int boid_blocks)
{
    if ((int)blockIdx.x < boid_blocks) {
        const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
        if (b < a.sc.nb_all && !(a.bmask && !a.bmask[b]))  // uniform per warp
            boid_fb_warp<false>(b, threadIdx.x & 31, a.pos, a.vel, a.rho, a.ab, a.start, a.sc, a.slot_of_boid,
                                a.bmask, a.fb, a.acc);
        return;
    }
    // particles base + lane, base stepping over the fluid blocks' threads; the
    // trip count is the block's, so every lane of a warp takes part in each
    // call (force_particle's warp-aggregated count)
    const int T = ((int)gridDim.x - boid_blocks) * (int)blockDim.x;
    for (int base = ((int)blockIdx.x - boid_blocks) * (int)blockDim.x; base < a.sc.n_all; base += T)
        force_particle<false>(a, base + (int)threadIdx.x);
}

cudaError_t launch_forces(const float4* pos, const SoaPos& xyz, const float4* vel, const float* rho, const float2* ab,
                          const float4* prec, const unsigned* start, const uint2* seg, const int* nseg,
                          const Scenes& sc,
                          const Tuning& t, const unsigned* list, const unsigned* list_off, size_t list_cap,
                          bool boids, bool fluid, const int* slot_of_boid, const int* bmask, float4* fb,
                          float4* acc, int* touched, float4* infl, float4* pos_next, float4* vel_next,
                          unsigned* key, unsigned* rank, unsigned* count, unsigned* err, cudaStream_t s,
                          long long* launches)
{
    const unsigned cap = list_cap > 0xffffffffu ? 0xffffffffu : (unsigned)list_cap;
    const int warps = t.block / 32;
    const int boid_blocks = boids ? (sc.nb_all + warps - 1) / warps : 0;
    const int per_block = t.block * (t.ppt > 1 ? t.ppt : 1);
    const int fluid_blocks = fluid ? (sc.n_all + per_block - 1) / per_block : 0;
    if (boid_blocks + fluid_blocks == 0) return cudaSuccess;
    const ForceArgs a{pos, xyz, vel, rho, ab, prec, start, t.use_seg ? seg : nullptr, nseg, sc, list, list_off, cap,
                      slot_of_boid, bmask, fb, acc, touched, infl, pos_next, vel_next, key, rank, count, err};
    k_forces<<<boid_blocks + fluid_blocks, t.block, 0, s>>>(a, boid_blocks);
    ++*launches;
    return cudaGetLastError();
}

// ------------------------------------------------- fused neighbour pipeline

// Both neighbour passes of every scene in one cooperative launch (the
// batched step's persistent pass): all CTAs are resident and take work
// items from two atomic queues.  Phase A: tiles of `tile` consecutive
// sorted slots (a run of cells of one or more scenes; each particle is
// independent), the density pass.  Then a grid barrier: every CTA arrives
// and waits for the others, a bounded wait (about 2^31 SM clock cycles, a
// second) after which it sets SPH_DEV_TIMEOUT and returns.  Phase B: groups
// of boids (a warp per boid: F_b) first, then the tiles again: the force
// pass.  queue[0], queue[1]: the phases' item counters, queue[2]: barrier
// arrivals (zeroed before every launch).  skip_cta >= 0 is a test hook:
// that CTA does not arrive, so the others give up at their limit.  Results
// are bit for bit those of the two launches (same per-particle code).
struct PipeArgs {
    ForceArgs f;
    float* rho;
    float2* ab;
    float4* prec;
    int* nbr;
    uint2* seg;
    int* nseg;
    int* ncand;
    unsigned* queue;
    int tile;
    unsigned n_tiles, n_boid_items;
    int skip_cta;
};

constexpr long long BARRIER_CYCLES = 1ll << 31;

// Arrive (unless skip) and wait until `expected` CTAs have arrived, at most
// BARRIER_CYCLES; false (and SPH_DEV_TIMEOUT) when the wait gave up.  The
// fences order this CTA's writes before its arrival and the other CTAs'
// writes before this CTA's later loads.
__device__ __forceinline__ bool grid_barrier(unsigned* arrive, unsigned expected, bool skip, unsigned* err)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (!skip) atomicAdd(arrive, 1u);
        int ok = 1;
        const long long t0 = clock64();
        while (atomicAdd(arrive, 0u) < expected) {
            if (clock64() - t0 > BARRIER_CYCLES) {
                atomicOr(err, SPH_DEV_TIMEOUT);
                ok = 0;
                break;
            }
            __nanosleep(500);
        }
        s_ok = ok;
    }
    __syncthreads();
    __threadfence();
    return s_ok != 0;
}

template <bool SEG>
__global__ void __launch_bounds__(256)
k_nbr_pipeline(PipeArgs a)
{
    __shared__ unsigned s_item;
    const Scenes& sc = a.f.sc;
    const int n_all = sc.n_all;
    for (;;) {  // phase A: density
        if (threadIdx.x == 0) s_item = atomicAdd(&a.queue[0], 1u);
        __syncthreads();
        const unsigned it = s_item;
        __syncthreads();
        if (it >= a.n_tiles) break;
        const int base = (int)it * a.tile, end = min(base + a.tile, n_all);
        for (int i = base + (int)threadIdx.x; i < end; i += blockDim.x)
            density_at<SEG>(i, a.f.pos, a.f.vel, a.f.xyz, a.f.start, sc, a.rho, a.ab, a.prec, a.nbr, a.seg, a.nseg,
                            a.ncand, a.f.err);
    }
    if (!grid_barrier(a.queue + 2, gridDim.x, (int)blockIdx.x == a.skip_cta, a.f.err)) return;
    const int warps = blockDim.x >> 5;
    for (;;) {  // phase B: F_b of the boids, then the forces
        if (threadIdx.x == 0) s_item = atomicAdd(&a.queue[1], 1u);
        __syncthreads();
        const unsigned it = s_item;
        __syncthreads();
        if (it >= a.n_boid_items + a.n_tiles) break;
        if (it < a.n_boid_items) {
            const int b = (int)it * warps + (int)(threadIdx.x >> 5);
            if (b < sc.nb_all)  // uniform per warp
                boid_fb_warp<true>(b, threadIdx.x & 31, a.f.pos, a.f.vel, a.f.rho, a.f.ab, a.f.start, sc,
                                   a.f.slot_of_boid, nullptr, a.f.fb, a.f.acc);
        } else {
            const int base = (int)(it - a.n_boid_items) * a.tile, end = min(base + a.tile, n_all);
            for (int o = 0; o < a.tile; o += blockDim.x) {  // every lane takes part
                const int i = base + o + (int)threadIdx.x;
                force_particle<true>(a.f, i < end ? i : n_all);
            }
        }
    }
}

cudaError_t launch_nbr_pipeline(const float4* pos, const SoaPos& xyz, const float4* vel, const unsigned* start,
                                const Scenes& sc, const Tuning& t, float* rho, float2* ab, float4* prec, int* nbr,
                                uint2* seg, int* nseg, int* ncand, const int* slot_of_boid, float4* fb,
                                float4* acc, int* touched, float4* infl, float4* pos_next, float4* vel_next,
                                unsigned* key, unsigned* rank, unsigned* count, unsigned* queue, int skip_cta,
                                unsigned* err, cudaStream_t s, long long* launches)
{
    if (sc.n_all <= 0) return cudaSuccess;
    const int block = t.pipe_block;
    const int tile = t.pipe_tile;
    const bool use_seg = t.use_seg != 0;
    const ForceArgs f{pos, xyz, vel, rho, ab, prec, start, use_seg ? seg : nullptr, nseg, sc, nullptr, nullptr, 0u,
                      slot_of_boid, nullptr, fb, acc, touched, infl, pos_next, vel_next, key, rank, count, err};
    const unsigned n_tiles = (unsigned)((sc.n_all + tile - 1) / tile);
    const unsigned warps = (unsigned)(block / 32);
    const unsigned n_boid_items = ((unsigned)sc.nb_all + warps - 1) / warps;
    const PipeArgs a{f, rho, ab, prec, nbr, seg, nseg, ncand, queue, tile, n_tiles, n_boid_items, skip_cta};
    void* fn = use_seg ? (void*)k_nbr_pipeline<true> : (void*)k_nbr_pipeline<false>;
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, block, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const unsigned items = n_tiles + n_boid_items;
    unsigned grid = (unsigned)per_sm * (unsigned)sm_count();  // every CTA resident
    if (grid > items) grid = items;
    e = cudaMemsetAsync(queue, 0, 3 * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = use_seg ? cudaLaunchKernelEx(&cfg, k_nbr_pipeline<true>, a) : cudaLaunchKernelEx(&cfg, k_nbr_pipeline<false>, a);
    ++*launches;
    return e;
}

// ---------------------------------------------------------- pair lists

// list[off[i] ..] = the neighbours of particle i in walk order: every j != i
// with r2 < h2, except attached j for attached i (the density pass counted
// exactly these: off is the exclusive scan of its counts).  A list that
// would end beyond cap is not written (the force pass walks instead).
__global__ void __launch_bounds__(256)
k_fill_lists(const float4* __restrict__ pos, const unsigned* __restrict__ start, Scenes sc,
             const unsigned* __restrict__ off, unsigned* __restrict__ list, size_t cap, unsigned* __restrict__ err)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = i < sc.n_all;
    bool over = false;
    if (active) {
        const unsigned o0 = off[i], o1 = off[i + 1];
        over = o1 > cap;
        if (!over && o1 > o0) {
            const StepConst& c = sc.c[scene_of(sc.pbase, sc.S, (unsigned)i)];
            const int nb_all = sc.nb_all;
            const float4 pi = pos[i];
            const bool att_i = id_of(pi) < nb_all;
            unsigned k = o0;
            RowWalk walk(c.g, c.wg, start + c.c_base, pi.x, pi.y, pi.z);
            unsigned s0, s1;
            while (walk.next(s0, s1)) {
                for (unsigned j = s0; j < s1; ++j) {
                    if (j == (unsigned)i) continue;
                    const float4 pj = __ldg(pos + j);
                    if (att_i && id_of(pj) < nb_all) continue;
                    const float r2 = pair_r2(__fsub_rn(pj.x, pi.x), __fsub_rn(pj.y, pi.y), __fsub_rn(pj.z, pi.z));
                    if (r2 < c.h2 && k < o1) list[k++] = j;
                }
            }
        }
    }
    if (__any_sync(FULL, over) && (threadIdx.x & 31) == 0) atomicOr(err, SPH_DEV_LIST_OVERFLOW);
}

cudaError_t launch_fill_lists(const float4* pos, const unsigned* start, const Scenes& sc, const unsigned* off,
                              unsigned* list, size_t cap, unsigned* err, cudaStream_t s, long long* launches)
{
    if (sc.n_all <= 0) return cudaSuccess;
    k_fill_lists<<<(sc.n_all + 255) / 256, 256, 0, s>>>(pos, start, sc, off, list, cap, err);
    ++*launches;
    return cudaGetLastError();
}

// ------------------------------------------- fixed-capacity hash grid

// The hash grid of section "Neighborhood Search": every particle appends
// its index to its cell's bucket through an atomic per-cell counter; a
// bucket holds at most cap indices and the particles beyond are dropped
// (the grid is lossy where cells are crowded).  Slots of the sorted state;
// the order inside a bucket is the order of the atomics.
__global__ void __launch_bounds__(256)
k_bucket_insert(const float4* __restrict__ pos, Scenes sc, unsigned* __restrict__ tracker,
                unsigned* __restrict__ buckets, int cap)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= sc.n_all) return;
    const StepConst& c = sc.c[scene_of(sc.pbase, sc.S, (unsigned)i)];
    const float4 p = pos[i];
    bool cl = false;
    const unsigned key = (unsigned)c.c_base + cell_key(c.g, p.x, p.y, p.z, &cl);
    const unsigned slot = atomicAdd(tracker + key, 1u);
    if (slot < (unsigned)cap) buckets[(size_t)key * cap + slot] = (unsigned)i;
}

// Neighbour count of every particle (by id) through the buckets: the cells within
// ceil(h / d) of its own (the 27 cells at d = h), min(count, cap) entries
// each, the predicate and exclusions of the density pass (j != i, no pair
// of attached particles).  dropped += the entries the buckets lost.
__global__ void __launch_bounds__(256)
k_bucket_count(const float4* __restrict__ pos, const unsigned* __restrict__ start, Scenes sc,
               const unsigned* __restrict__ tracker, const unsigned* __restrict__ buckets, int cap,
               int* __restrict__ counts, unsigned long long* __restrict__ dropped)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= sc.n_all) return;
    const StepConst& c = sc.c[scene_of(sc.pbase, sc.S, (unsigned)i)];
    const float4 pi = pos[i];
    const bool att_i = id_of(pi) < sc.nb_all;
    bool cl = false;
    const int cx = cell_coord(pi.x, c.g.minf[0], c.g.inv_dx, c.g.dim[0], &cl);
    const int cy = cell_coord(pi.y, c.g.minf[1], c.g.inv_d, c.g.dim[1], &cl);
    const int cz = cell_coord(pi.z, c.g.minf[2], c.g.inv_d, c.g.dim[2], &cl);
    const int R = (int)ceilf(c.h * c.g.inv_d), Rx = (int)ceilf(c.h * c.g.inv_dx);
    int n = 0;
    for (int z = max(cz - R, 0); z <= min(cz + R, c.g.dim[2] - 1); ++z)
        for (int y = max(cy - R, 0); y <= min(cy + R, c.g.dim[1] - 1); ++y)
            for (int x = max(cx - Rx, 0); x <= min(cx + Rx, c.g.dim[0] - 1); ++x) {
                const unsigned key = (unsigned)c.c_base + (unsigned)x +
                                     (unsigned)c.g.dim[0] * ((unsigned)y + (unsigned)c.g.dim[1] * (unsigned)z);
                const unsigned m = min(__ldg(tracker + key), (unsigned)cap);
                for (unsigned k = 0; k < m; ++k) {
                    const unsigned j = __ldg(buckets + (size_t)key * cap + k);
                    if (j == (unsigned)i) continue;
                    const float4 pj = __ldg(pos + j);
                    if (att_i && id_of(pj) < sc.nb_all) continue;
                    if (pair_r2(__fsub_rn(pj.x, pi.x), __fsub_rn(pj.y, pi.y), __fsub_rn(pj.z, pi.z)) < c.h2) ++n;
                }
            }
    counts[id_of(pi)] = n;
    // the first slot of each cell (sorted order) reports what the cell lost
    const unsigned own = (unsigned)c.c_base + (unsigned)cx +
                         (unsigned)c.g.dim[0] * ((unsigned)cy + (unsigned)c.g.dim[1] * (unsigned)cz);
    const unsigned t = tracker[own];
    if (t > (unsigned)cap && (unsigned)i == __ldg(start + own))
        atomicAdd(dropped, (unsigned long long)(t - (unsigned)cap));
}

cudaError_t launch_bucket_neighbors(const float4* pos, const unsigned* start, const Scenes& sc, unsigned* tracker,
                                    int ncells,
                                    unsigned* buckets, int cap, int* counts, unsigned long long* dropped,
                                    cudaStream_t s, long long* launches)
{
    if (sc.n_all <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(tracker, 0, (size_t)ncells * sizeof(unsigned), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(dropped, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    const int blocks = (sc.n_all + 255) / 256;
    k_bucket_insert<<<blocks, 256, 0, s>>>(pos, sc, tracker, buckets, cap);
    k_bucket_count<<<blocks, 256, 0, s>>>(pos, start, sc, tracker, buckets, cap, counts, dropped);
    *launches += 2;
    return cudaGetLastError();
}

// ---------------------------------------------------------- neighbour list

__global__ void __launch_bounds__(256)
k_neighbor_list(const float4* __restrict__ pos, const unsigned* __restrict__ start, Scenes sc,
                int* __restrict__ counts, const long long* __restrict__ offsets, int* __restrict__ list)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= sc.n_all) return;
    const StepConst& c = sc.c[scene_of(sc.pbase, sc.S, (unsigned)i)];
    const float4 pi = pos[i];
    const int id_i = id_of(pi);
    const bool att_i = id_i < sc.nb_all;
    long long o = offsets ? offsets[id_i] : 0;
    int cnt = 0;
    RowWalk walk(c.g, c.wg, start + c.c_base, pi.x, pi.y, pi.z);
    unsigned s0, s1;
    while (walk.next(s0, s1)) {
        for (unsigned j = s0; j < s1; ++j) {
            if (j == (unsigned)i) continue;
            const float4 pj = pos[j];
            if (att_i && id_of(pj) < sc.nb_all) continue;
            float r2 = pair_r2(__fsub_rn(pj.x, pi.x), __fsub_rn(pj.y, pi.y), __fsub_rn(pj.z, pi.z));
            if (r2 < c.h2) {
                if (list) list[o + cnt] = id_of(pj);
                ++cnt;
            }
        }
    }
    counts[id_i] = cnt;
}

cudaError_t launch_neighbor_list(const float4* pos, const unsigned* start, const Scenes& sc, int* counts,
                                 const long long* offsets, int* list, cudaStream_t s, long long* launches)
{
    if (sc.n_all <= 0) return cudaSuccess;
    k_neighbor_list<<<(sc.n_all + 255) / 256, 256, 0, s>>>(pos, start, sc, counts, offsets, list);
    ++*launches;
    return cudaGetLastError();
}

}  // namespace sphk
