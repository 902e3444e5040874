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
// One block of FT threads per boid sweeps the particle-grid rows under the
// stencil's box (one cell of margin) once: counts and velocity sums go to
// shared bins by integer atomics (velocities in 2^-32 fixed point, so the
// sums do not depend on the order), the kernel moments to per-thread sums
// reduced in a fixed order.
#include <cuda_bf16.h>

#include "sph_internal.cuh"

namespace sphk {

constexpr int FT = 128;
constexpr double FIX = 4294967296.0;  // 2^32

__global__ void __launch_bounds__(FT)
k_features(const float4* __restrict__ pos, const float4* __restrict__ vel, const unsigned* __restrict__ start,
           const float4* __restrict__ bpos, const float4* __restrict__ bvel, Scenes sc,
           __nv_bfloat16* __restrict__ x)
{
    __shared__ int cnt[64];
    __shared__ unsigned long long vsum[64][3];
    __shared__ float red[FT / 32][10];
    const int b = blockIdx.x;
    const int tid = threadIdx.x;
    const StepConst& c = sc.c[scene_of(sc.bbase, sc.S, (unsigned)b)];
    const float4 pb = bpos[b], vb = bvel[b];
    const float p[3] = {pb.x, pb.y, pb.z};
    float c0[3], centre_off[3];
    int lo[3], hi[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float t = __fmul_rn(__fsub_rn(p[a], c.g.minf[a]), c.inv_h);
        c0[a] = floorf(__fsub_rn(t, 1.5f));
        centre_off[a] = __fsub_rn(__fsub_rn(t, c0[a]), 2.0f);
        // particle-grid cells under [c0 h, (c0 + 4) h) (relative to m), +-1 cell
        const float e0 = __fmul_rn(__fmul_rn(c0[a], c.h), c.g.inv_d);
        const float e1 = __fmul_rn(__fmul_rn(c0[a] + 4.0f, c.h), c.g.inv_d);
        lo[a] = (int)fmaxf(floorf(e0) - 1.0f, 0.0f);
        hi[a] = (int)fminf(floorf(e1) + 1.0f, (float)(c.g.dim[a] - 1));
    }
    if (tid < 64) {
        cnt[tid] = 0;
        vsum[tid][0] = vsum[tid][1] = vsum[tid][2] = 0ull;
    }
    __syncthreads();
    const float h2 = c.h2;
    float m[10] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // poly6, S0, S1 (3), S2 (3)
    const unsigned* cstart = start + c.c_base;
    for (int z = lo[2]; z <= hi[2]; ++z) {
        for (int y = lo[1]; y <= hi[1]; ++y) {
            if (lo[0] > hi[0]) continue;
            const unsigned row = (unsigned)c.g.dim[0] * ((unsigned)y + (unsigned)c.g.dim[1] * (unsigned)z);
            const unsigned s0 = __ldg(cstart + row + lo[0]), s1 = __ldg(cstart + row + hi[0] + 1);
            for (unsigned j = s0 + tid; j < s1; j += FT) {
                const float4 pj = __ldg(pos + j);
                if (id_of(pj) < sc.nb_all) continue;  // fluid particles only
                const float fx = floorf(__fmul_rn(__fsub_rn(pj.x, c.g.minf[0]), c.inv_h)) - c0[0];
                const float fy = floorf(__fmul_rn(__fsub_rn(pj.y, c.g.minf[1]), c.inv_h)) - c0[1];
                const float fz = floorf(__fmul_rn(__fsub_rn(pj.z, c.g.minf[2]), c.inv_h)) - c0[2];
                const bool in = fx >= 0.f && fx < 4.f && fy >= 0.f && fy < 4.f && fz >= 0.f && fz < 4.f;
                const float dx = __fsub_rn(pj.x, pb.x), dy = __fsub_rn(pj.y, pb.y), dz = __fsub_rn(pj.z, pb.z);
                const float r2 = pair_r2(dx, dy, dz);
                const bool near = r2 < h2;
                if (!in && !near) continue;
                const float4 vj = __ldg(vel + j);
                if (in) {
                    const int q = (int)fx + 4 * ((int)fy + 4 * (int)fz);
                    atomicAdd(&cnt[q], 1);
                    atomicAdd(&vsum[q][0], (unsigned long long)__double2ll_rn((double)vj.x * FIX));
                    atomicAdd(&vsum[q][1], (unsigned long long)__double2ll_rn((double)vj.y * FIX));
                    atomicAdd(&vsum[q][2], (unsigned long long)__double2ll_rn((double)vj.z * FIX));
                }
                if (near) {
                    const float u = h2 - r2;
                    m[0] += u * u * u;
                    const float r = sqrtf(r2);
                    const float w = 1.0f - r * c.inv_h;
                    m[1] += w;
                    m[2] += w * (vj.x - vb.x);
                    m[3] += w * (vj.y - vb.y);
                    m[4] += w * (vj.z - vb.z);
                    if (r2 > 0.0f) {
                        const float s = -w * w / r;  // (x_b - x_j) / r = -d / r
                        m[5] += s * dx;
                        m[6] += s * dy;
                        m[7] += s * dz;
                    }
                }
            }
        }
    }
    // fixed-order reduction of the moments: warp butterflies, then warps in order
#pragma unroll
    for (int k = 0; k < 8; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m[k] += __shfl_xor_sync(FULL, m[k], o);
    }
    if ((tid & 31) == 0) {
#pragma unroll
        for (int k = 0; k < 8; ++k) red[tid >> 5][k] = m[k];
    }
    __syncthreads();
    __nv_bfloat16* row = x + (size_t)b * SPH_MLP_IN;
    if (tid < 64) {
        const int n = cnt[tid];
        const float dens = (float)n * (c.mass / (c.h * c.h * c.h * c.rho0));
        const double inv = n ? 1.0 / ((double)n * FIX) : 0.0;
        row[4 * tid + 0] = __float2bfloat16_rn(dens);
        row[4 * tid + 1] = __float2bfloat16_rn((float)((double)(long long)vsum[tid][0] * inv));
        row[4 * tid + 2] = __float2bfloat16_rn((float)((double)(long long)vsum[tid][1] * inv));
        row[4 * tid + 3] = __float2bfloat16_rn((float)((double)(long long)vsum[tid][2] * inv));
    } else if (tid < 64 + (SPH_MLP_IN - 256)) {
        const int k = tid - 64;
        float tot[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            float acc = 0.0f;
            for (int w = 0; w < FT / 32; ++w) acc += red[w][i];
            tot[i] = acc;
        }
        const float kn = c.mass / (c.rho0 * c.h * c.h * c.h);
        float v = 0.0f;
        if (k < 3) v = k == 0 ? vb.x : (k == 1 ? vb.y : vb.z);
        else if (k < 6) v = centre_off[k - 3];
        else if (k == 6) v = c.mC6 * (tot[0] + h2 * h2 * h2) / c.rho0;
        else if (k < 14) v = kn * tot[k - 6];
        row[256 + k] = __float2bfloat16_rn(v);
    }
}

cudaError_t launch_features(const float4* pos, const float4* vel, const unsigned* start, const float4* bpos,
                            const float4* bvel, const Scenes& sc, void* x, cudaStream_t s, long long* launches)
{
    if (sc.nb_all <= 0) return cudaSuccess;
    k_features<<<sc.nb_all, FT, 0, s>>>(pos, vel, start, bpos, bvel, sc, (__nv_bfloat16*)x);
    ++*launches;
    return cudaGetLastError();
}

// For every attached particle whose boid is flagged (bmask NULL = all):
// need[slot] = 1 for the particle and for each fluid neighbour (their
// densities enter the boid's force).
__global__ void __launch_bounds__(256)
k_mark_needed(const float4* __restrict__ pos, const unsigned* __restrict__ start, Scenes sc,
              const int* __restrict__ bmask, unsigned char* __restrict__ need)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= sc.n_all) return;
    const float4 pi = pos[i];
    const int id = id_of(pi);
    if (id >= sc.nb_all || (bmask && !bmask[id])) return;
    need[i] = 1;
    const StepConst& c = sc.c[scene_of(sc.pbase, sc.S, (unsigned)i)];
    RowWalk walk(c.g, c.wg, start + c.c_base, pi.x, pi.y, pi.z);
    unsigned s0, s1;
    while (walk.next(s0, s1)) {
        for (unsigned j = s0; j < s1; ++j) {
            const float4 pj = pos[j];
            if (id_of(pj) < sc.nb_all) continue;
            const float r2 = pair_r2(__fsub_rn(pj.x, pi.x), __fsub_rn(pj.y, pi.y), __fsub_rn(pj.z, pi.z));
            if (r2 < c.h2) need[j] = 1;
        }
    }
}

cudaError_t launch_mark_needed(const float4* pos, const unsigned* start, const Scenes& sc, const int* bmask,
                               unsigned char* need, cudaStream_t s, long long* launches)
{
    if (sc.n_all <= 0) return cudaSuccess;
    k_mark_needed<<<(sc.n_all + 255) / 256, 256, 0, s>>>(pos, start, sc, bmask, need);
    ++*launches;
    return cudaGetLastError();
}

// Network output y [nb][16] -> forces: F_b = y[0:3] * f_scale, w = 0; the
// boid is flagged for the exact path (flag = 1) where the error head
// y[3] (log10 of the expected relative error) exceeds log_err_max or the
// output is not finite.
__global__ void k_surrogate_out(const float* __restrict__ y, int nb, float f_scale, float log_err_max,
                                float4* __restrict__ out, int* __restrict__ flag, unsigned* __restrict__ nflag)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    const float* r = y + (size_t)b * SPH_MLP_OUT;
    const float fx = r[0] * f_scale, fy = r[1] * f_scale, fz = r[2] * f_scale;
    const bool bad = !(r[3] <= log_err_max) || !isfinite(fx) || !isfinite(fy) || !isfinite(fz);
    out[b] = make_float4(fx, fy, fz, 0.0f);
    flag[b] = bad ? 1 : 0;
    if (bad && nflag) atomicAdd(nflag, 1u);
}

cudaError_t launch_surrogate_out(const float* y, int nb, float f_scale, float log_err_max, float4* out, int* flag,
                                 unsigned* nflag, cudaStream_t s, long long* launches)
{
    if (nb <= 0) return cudaSuccess;
    k_surrogate_out<<<(nb + 255) / 256, 256, 0, s>>>(y, nb, f_scale, log_err_max, out, flag, nflag);
    ++*launches;
    return cudaGetLastError();
}

}  // namespace sphk
