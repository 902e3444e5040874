// sph_features.cu -- the inputs and outputs of the boid-force surrogate on
// the sorted state: the stencil features of every boid, the marking of the
// particles whose density an exact fluid force on a boid needs, and the
// conversion of the network output into forces with the error gate.
//
// Features of boid b: one row of 272 BF16.
//   0 .. 255  the 4 x 4 x 4 cells of size h of a feature grid anchored at
//             the box minimum m, starting at c0 = floor((p_b - m) / h - 1.5)
//             per axis (the boid lies in the central 2 x 2 x 2 cells, at
//             least 1.5 h from the stencil's faces, so the stencil holds its
//             whole h-sphere); cell q = (iz * 4 + iy) * 4 + ix gives columns
//             4q .. 4q+3 = (fluid count * m / (h^3 rho0), mean fluid velocity)
//   256 .. 258  the boid's velocity
//   259 .. 261  its offset from the stencil's centre, (p_b - m) / h - c0 - 2,
//               in [-0.5, 0.5)
//   262       rho_b / rho0: the SPH density of the boid's attached particle
//             (self term + fluid neighbours, as in the step)
//   263       S0 = m / (rho0 h^3) sum_j (1 - q)
//   264 .. 266  S1 = m / (rho0 h^3) sum_j (1 - q) (v_j - v_b)
//   267 .. 269  S2 = m / (rho0 h^3) sum_j (1 - q)^2 (x_b - x_j) / r
//   270, 271  zero
// with j over the fluid particles within h of the boid and q = r / h.
// Cells outside the grid contribute zeros.  A feature cell of a particle is
// floor((x - m) * inv_h) in float32 (inv_h = fl(1 / h)), like the grid's
// own cell function.
//
#include <cuda_bf16.h>

#include "sph_internal.cuh"

namespace sphk {

// Stencil features in two launches:
//   1. k_feature_grid (K8): every fluid particle adds 1 and its velocity (in
//      2^-16 fixed point) to the integer sums of its feature cell, kept for
//      the box plus two cells of margin on every side (a boid in the box
//      has its whole stencil there; integer sums do not depend on the
//      order, and they hold while a cell's mean speed stays below
//      2^15 / count m/s, beyond any flow of these scenes);
//   2. k_features (K9): a warp per boid reads its 4 x 4 x 4 cells from the
//      grid (cells outside it are zeros) and walks the particle grid around
//      it for the kernel moments (WarpRows: the lanes take the walk's
//      candidates by flat index, each keeping its own sums, then a
//      butterfly adds the 32 sums in a fixed order).
constexpr float VFIX = 65536.0f;
constexpr int FW = 8;  // warps per block of k_features

__global__ void __launch_bounds__(256)
k_feature_grid(const float4* __restrict__ pos, const float4* __restrict__ vel, Scenes sc, int4* __restrict__ grid)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned lane = threadIdx.x & 31u;
    int q = -1;  // feature cell of this lane's particle, -1: none
    int4 v = make_int4(0, 0, 0, 0);
    if (i < sc.n_all) {
        const float4 p = pos[i];
        if (id_of(p) >= sc.nb_all) {  // fluid particles only
            const StepConst& c = sc.c[scene_of(sc.pbase, sc.S, (unsigned)i)];
            // feature cell floor((x - m) inv_h), shifted by the two-cell margin
            const float fx = floorf(__fmul_rn(__fsub_rn(p.x, c.g.minf[0]), c.inv_h)) + 2.0f;
            const float fy = floorf(__fmul_rn(__fsub_rn(p.y, c.g.minf[1]), c.inv_h)) + 2.0f;
            const float fz = floorf(__fmul_rn(__fsub_rn(p.z, c.g.minf[2]), c.inv_h)) + 2.0f;
            // more than two cells outside the box: no boid of the box sees it
            if (fx >= 0.f && fx < (float)c.fdim[0] && fy >= 0.f && fy < (float)c.fdim[1] && fz >= 0.f &&
                fz < (float)c.fdim[2]) {
                q = c.fc_base + (int)fx + c.fdim[0] * ((int)fy + c.fdim[1] * (int)fz);
                const float4 u = __ldg(vel + i);
                v = make_int4(1, __float2int_rn(u.x * VFIX), __float2int_rn(u.y * VFIX), __float2int_rn(u.z * VFIX));
            }
        }
    }
    // Consecutive sorted particles mostly share a cell: the lanes of a run
    // of equal q add their sums (integer prefix sums of the warp, the run's
    // sum = the prefix at its last lane minus the prefix before its first)
    // and the run's last lane adds them to the grid.
    const int qp = __shfl_up_sync(FULL, q, 1);
    const unsigned heads = __ballot_sync(FULL, lane == 0 || qp != q);
    int4 incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int a = __shfl_up_sync(FULL, incl.x, o), b = __shfl_up_sync(FULL, incl.y, o);
        const int c = __shfl_up_sync(FULL, incl.z, o), d = __shfl_up_sync(FULL, incl.w, o);
        if (lane >= (unsigned)o) {
            incl.x += a;
            incl.y += b;
            incl.z += c;
            incl.w += d;
        }
    }
    const int head = 31 - __clz(heads & (0xffffffffu >> (31u - lane)));  // first lane of this lane's run
    const int src = head > 0 ? head - 1 : 0;
    int4 before = make_int4(__shfl_sync(FULL, incl.x, src), __shfl_sync(FULL, incl.y, src),
                            __shfl_sync(FULL, incl.z, src), __shfl_sync(FULL, incl.w, src));
    if (head == 0) before = make_int4(0, 0, 0, 0);
    const bool tail = lane == 31u || ((heads >> (lane + 1u)) & 1u);
    if (tail && q >= 0) {
        atomicAdd(&grid[q].x, incl.x - before.x);
        atomicAdd(&grid[q].y, incl.y - before.y);
        atomicAdd(&grid[q].z, incl.z - before.z);
        atomicAdd(&grid[q].w, incl.w - before.w);
    }
}

__global__ void __launch_bounds__(FW * 32)
k_features(const float4* __restrict__ pos, const float4* __restrict__ vel, const unsigned* __restrict__ start,
           const float4* __restrict__ bpos, const float4* __restrict__ bvel, Scenes sc,
           const int4* __restrict__ grid, __nv_bfloat16* __restrict__ x)
{
    const int lane = threadIdx.x & 31;
    const int b = blockIdx.x * FW + (int)(threadIdx.x >> 5);
    if (b >= sc.nb_all) return;  // the whole warp
    const StepConst& c = sc.c[scene_of(sc.bbase, sc.S, (unsigned)b)];
    const float4 pb = bpos[b], vb = bvel[b];
    const float p[3] = {pb.x, pb.y, pb.z};
    float c0[3], centre_off[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float t = __fmul_rn(__fsub_rn(p[a], c.g.minf[a]), c.inv_h);
        c0[a] = floorf(__fsub_rn(t, 1.5f));
        centre_off[a] = __fsub_rn(__fsub_rn(t, c0[a]), 2.0f);
    }
    __nv_bfloat16* row = x + (size_t)b * SPH_MLP_IN;
    // ---- the 64 stencil cells from the grid (two per lane)
    const float dens_unit = c.mass / (c.h * c.h * c.h * c.rho0);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int q = lane + 32 * k;
        const float gx = c0[0] + (float)(q & 3) + 2.0f, gy = c0[1] + (float)((q >> 2) & 3) + 2.0f,
                    gz = c0[2] + (float)(q >> 4) + 2.0f;
        int4 v = make_int4(0, 0, 0, 0);
        if (gx >= 0.f && gx < (float)c.fdim[0] && gy >= 0.f && gy < (float)c.fdim[1] && gz >= 0.f &&
            gz < (float)c.fdim[2])
            v = __ldg(grid + c.fc_base + (int)gx + c.fdim[0] * ((int)gy + c.fdim[1] * (int)gz));
        const float inv = v.x ? 1.0f / ((float)v.x * VFIX) : 0.0f;
        row[4 * q + 0] = __float2bfloat16_rn((float)v.x * dens_unit);
        row[4 * q + 1] = __float2bfloat16_rn((float)v.y * inv);
        row[4 * q + 2] = __float2bfloat16_rn((float)v.z * inv);
        row[4 * q + 3] = __float2bfloat16_rn((float)v.w * inv);
    }
    // ---- kernel moments over the fluid particles within h of the boid
    const float h2 = c.h2;
    float mo[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // poly6, S0, S1 (3), S2 (3)
    WarpRows rows(c.g, c.wg, start + c.c_base, pb.x, pb.y, pb.z);
    for (int bt = 0; 32 * bt < rows.nrows; ++bt) {
        rows.batch(bt);
        const unsigned total = rows.flatten();
        for (unsigned k0 = 0; k0 < total; k0 += 32) {
            const unsigned k = k0 + (unsigned)lane;
            const unsigned j = rows.slot(k < total ? k : total - 1);
            if (k >= total) continue;
            const float4 pj = __ldg(pos + j);
            if (id_of(pj) < sc.nb_all) continue;  // fluid particles only
            const float dx = __fsub_rn(pj.x, pb.x), dy = __fsub_rn(pj.y, pb.y), dz = __fsub_rn(pj.z, pb.z);
            const float r2 = pair_r2(dx, dy, dz);
            if (r2 < h2) {
                const float4 vj = __ldg(vel + j);
                const float u2 = h2 - r2;
                mo[0] += u2 * u2 * u2;
                const float rr = sqrtf(r2);
                const float w = 1.0f - rr * c.inv_h;
                mo[1] += w;
                mo[2] += w * (vj.x - vb.x);
                mo[3] += w * (vj.y - vb.y);
                mo[4] += w * (vj.z - vb.z);
                if (r2 > 0.0f) {
                    const float sdir = -w * w / rr;  // (x_b - x_j) / r = -d / r
                    mo[5] += sdir * dx;
                    mo[6] += sdir * dy;
                    mo[7] += sdir * dz;
                }
            }
        }
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mo[k] += __shfl_xor_sync(FULL, mo[k], o);
    }
    if (lane < SPH_MLP_IN - 256) {
        const int m = lane;
        const float kn = c.mass / (c.rho0 * c.h * c.h * c.h);
        float v = 0.0f;
        if (m < 3) v = m == 0 ? vb.x : (m == 1 ? vb.y : vb.z);
        else if (m < 6) v = centre_off[m - 3];
        else if (m == 6) v = c.mC6 * (mo[0] + h2 * h2 * h2) / c.rho0;
        else if (m < 14) v = kn * mo[m - 6];
        row[256 + m] = __float2bfloat16_rn(v);
    }
}

cudaError_t launch_features(const float4* pos, const float4* vel, const unsigned* start, const float4* bpos,
                            const float4* bvel, const Scenes& sc, int4* grid, int nfcells, void* x, cudaStream_t s,
                            long long* launches)
{
    if (sc.nb_all <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(grid, 0, (size_t)nfcells * sizeof(int4), s);
    if (e != cudaSuccess) return e;
    if (sc.n_all > 0) {
        k_feature_grid<<<(sc.n_all + 255) / 256, 256, 0, s>>>(pos, vel, sc, grid);
        ++*launches;
    }
    k_features<<<(sc.nb_all + FW - 1) / FW, FW * 32, 0, s>>>(pos, vel, start, bpos, bvel, sc, grid,
                                                              (__nv_bfloat16*)x);
    ++*launches;
    return cudaGetLastError();
}

// For every flagged boid (bmask NULL = all): need[slot] = 1 for its attached
// particle and for each fluid neighbour (their densities enter the boid's
// force).  One warp per boid: the lanes fetch the walk's rows together
// (WarpRows) and take the candidates by flat index.
constexpr int MARK_WARPS = 8;

__global__ void __launch_bounds__(MARK_WARPS * 32)
k_mark_needed(const float4* __restrict__ pos, const unsigned* __restrict__ start, Scenes sc,
              const int* __restrict__ slot_of_boid, const int* __restrict__ bmask, unsigned char* __restrict__ need)
{
    const int b = blockIdx.x * MARK_WARPS + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (b >= sc.nb_all || (bmask && !bmask[b])) return;  // uniform per warp
    const int i = slot_of_boid[b];
    if (lane == 0) need[i] = 1;
    const float4 pi = pos[i];
    const StepConst& c = sc.c[scene_of(sc.pbase, sc.S, (unsigned)i)];
    WarpRows rows(c.g, c.wg, start + c.c_base, pi.x, pi.y, pi.z);
    for (int bt = 0; 32 * bt < rows.nrows; ++bt) {
        rows.batch(bt);
        const unsigned total = rows.flatten();
        for (unsigned k0 = 0; k0 < total; k0 += 32) {
            const unsigned k = k0 + (unsigned)lane;
            const unsigned j = rows.slot(k < total ? k : total - 1);
            if (k >= total) continue;
            const float4 pj = __ldg(pos + j);
            if (id_of(pj) < sc.nb_all) continue;
            const float r2 = pair_r2(__fsub_rn(pj.x, pi.x), __fsub_rn(pj.y, pi.y), __fsub_rn(pj.z, pi.z));
            if (r2 < c.h2) need[j] = 1;
        }
    }
}

cudaError_t launch_mark_needed(const float4* pos, const unsigned* start, const Scenes& sc, const int* slot_of_boid,
                               const int* bmask, unsigned char* need, cudaStream_t s, long long* launches)
{
    if (sc.nb_all <= 0) return cudaSuccess;
    k_mark_needed<<<(sc.nb_all + MARK_WARPS - 1) / MARK_WARPS, MARK_WARPS * 32, 0, s>>>(pos, start, sc, slot_of_boid,
                                                                                          bmask, need);
    ++*launches;
    return cudaGetLastError();
}

// Stream compaction of the marked slots: one atomic per warp.
__global__ void __launch_bounds__(256)
k_compact_needed(const unsigned char* __restrict__ need, int n, int* __restrict__ list, unsigned* __restrict__ len)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool take = i < n && need[i];
    const unsigned ballot = __ballot_sync(FULL, take);
    if (!ballot) return;
    const int lane = threadIdx.x & 31;
    unsigned base = 0;
    if (lane == 0) base = atomicAdd(len, (unsigned)__popc(ballot));
    base = __shfl_sync(FULL, base, 0);
    if (take) list[base + __popc(ballot & ((1u << lane) - 1u))] = i;
}

cudaError_t launch_compact_needed(const unsigned char* need, int n, int* list, unsigned* len, cudaStream_t s,
                                  long long* launches)
{
    cudaError_t e = cudaMemsetAsync(len, 0, sizeof(unsigned), s);
    if (e != cudaSuccess || n <= 0) return e;
    k_compact_needed<<<(n + 255) / 256, 256, 0, s>>>(need, n, list, len);
    ++*launches;
    return cudaGetLastError();
}

// Network output y [nb][16] -> forces: F_b = y[0:3] * f_scale, w = 0; the
// boid is flagged for the exact path (flag = 1) where the error head
// y[3] (log10 of the expected relative error) exceeds log_err_max, the
// output is not finite, or (lo, hi given) a feature lies outside [lo, hi].
// A warp per boid: the lanes test the row's 34 chunks of 8 BF16 features.
constexpr int SO_THREADS = 256;

__global__ void __launch_bounds__(SO_THREADS) k_surrogate_out(
    const float* __restrict__ y, const __nv_bfloat16* __restrict__ x, const float* __restrict__ lo,
    const float* __restrict__ hi, int nb, float f_scale, float log_err_max, float4* __restrict__ out,
    int* __restrict__ flag, unsigned* __restrict__ nflag)
{
    const int b = (int)(((size_t)blockIdx.x * SO_THREADS + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (b >= nb) return;  // the whole warp
    bool oob = false;
    if (lo) {
        static_assert(SPH_MLP_IN % 8 == 0, "rows are whole 16-byte chunks");
        const uint4* row = reinterpret_cast<const uint4*>(x + (size_t)b * SPH_MLP_IN);
        for (int c = lane; c < SPH_MLP_IN / 8; c += 32) {
            const uint4 v = __ldg(row + c);
            const unsigned w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                // BF16 -> FP32 is the high half of the word
                const float a = __uint_as_float(w[j] << 16), e = __uint_as_float(w[j] & 0xffff0000u);
                const int k = c * 8 + 2 * j;
                oob |= !(a >= __ldg(lo + k) && a <= __ldg(hi + k));
                oob |= !(e >= __ldg(lo + k + 1) && e <= __ldg(hi + k + 1));
            }
        }
        oob = __any_sync(0xffffffffu, oob);
    }
    if (lane != 0) return;
    const float* r = y + (size_t)b * SPH_MLP_OUT;
    const float fx = r[0] * f_scale, fy = r[1] * f_scale, fz = r[2] * f_scale;
    const bool bad = oob || !(r[3] <= log_err_max) || !isfinite(fx) || !isfinite(fy) || !isfinite(fz);
    out[b] = make_float4(fx, fy, fz, 0.0f);
    flag[b] = bad ? 1 : 0;
    if (bad && nflag) atomicAdd(nflag, 1u);
}

cudaError_t launch_surrogate_out(const float* y, const void* x, const float* lo, const float* hi, int nb,
                                 float f_scale, float log_err_max, float4* out, int* flag, unsigned* nflag,
                                 cudaStream_t s, long long* launches)
{
    if (nb <= 0) return cudaSuccess;
    const int per_block = SO_THREADS / 32;
    k_surrogate_out<<<(nb + per_block - 1) / per_block, SO_THREADS, 0, s>>>(
        y, (const __nv_bfloat16*)x, lo, hi, nb, f_scale, log_err_max, out, flag, nflag);
    ++*launches;
    return cudaGetLastError();
}

}  // namespace sphk
