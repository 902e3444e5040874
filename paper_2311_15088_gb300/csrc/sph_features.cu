// sph_features.cu -- the inputs and outputs of the boid-force surrogate on
// the sorted state: the stencil features of every boid, the marking of the
// particles whose density an exact fluid force on a boid needs, and the
// conversion of the network output into forces with the error gate.
//
// Features of boid b (one row of 272 BF16): the 4 x 4 x 4 cells of the
// particle grid starting at c0 = floor((p_b - m) / d - 1.5) per axis (the
// boid lies in the central 2 x 2 x 2 cells); cell q = (iz * 4 + iy) * 4 + ix
// gives columns 4q .. 4q+3 = (fluid count * m / (d^3 rho0), mean fluid
// velocity); columns 256 .. 258 are the boid's velocity; the rest are zero.
// Cells outside the grid contribute zeros.
#include <cuda_bf16.h>

#include "sph_internal.cuh"

namespace sphk {

__global__ void __launch_bounds__(64)
k_features(const float4* __restrict__ pos, const float4* __restrict__ vel, const unsigned* __restrict__ start,
           const float4* __restrict__ bpos, const float4* __restrict__ bvel, Scenes sc,
           __nv_bfloat16* __restrict__ x)
{
    const int b = blockIdx.x;
    const int q = threadIdx.x;
    const StepConst& c = sc.c[scene_of(sc.bbase, sc.S, (unsigned)b)];
    const float4 pb = bpos[b];
    const float p[3] = {pb.x, pb.y, pb.z};
    const int off[3] = {q & 3, (q >> 2) & 3, q >> 4};
    int cell[3];
    bool inside = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float t = __fmul_rn(__fsub_rn(p[a], c.g.minf[a]), c.g.inv_d);
        const float c0 = floorf(__fsub_rn(t, 1.5f));
        // stencil origins far outside the grid cannot reach it
        const float ca = c0 + (float)off[a];
        inside = inside && ca >= 0.0f && ca <= (float)(c.g.dim[a] - 1);
        cell[a] = inside ? (int)ca : 0;
    }
    int count = 0;
    float sx = 0.f, sy = 0.f, sz = 0.f;
    if (inside) {
        const unsigned key = (unsigned)c.c_base + (unsigned)cell[0] +
                             (unsigned)c.g.dim[0] * ((unsigned)cell[1] + (unsigned)c.g.dim[1] * (unsigned)cell[2]);
        for (unsigned j = start[key]; j < start[key + 1]; ++j) {
            if (id_of(pos[j]) < sc.nb_all) continue;  // fluid particles only
            const float4 v = vel[j];
            ++count;
            sx += v.x;
            sy += v.y;
            sz += v.z;
        }
    }
    const float d = c.wg.d;
    const float dens = (float)count * (c.mass / (d * d * d * c.rho0));
    const float inv = count ? 1.0f / (float)count : 0.0f;
    __nv_bfloat16* row = x + (size_t)b * SPH_MLP_IN;
    row[4 * q + 0] = __float2bfloat16_rn(dens);
    row[4 * q + 1] = __float2bfloat16_rn(sx * inv);
    row[4 * q + 2] = __float2bfloat16_rn(sy * inv);
    row[4 * q + 3] = __float2bfloat16_rn(sz * inv);
    if (q < SPH_MLP_IN - 256) {
        const float4 vb = bvel[b];
        const float v = q == 0 ? vb.x : (q == 1 ? vb.y : (q == 2 ? vb.z : 0.0f));
        row[256 + q] = __float2bfloat16_rn(v);
    }
}

cudaError_t launch_features(const float4* pos, const float4* vel, const unsigned* start, const float4* bpos,
                            const float4* bvel, const Scenes& sc, void* x, cudaStream_t s, long long* launches)
{
    if (sc.nb_all <= 0) return cudaSuccess;
    k_features<<<sc.nb_all, 64, 0, s>>>(pos, vel, start, bpos, bvel, sc, (__nv_bfloat16*)x);
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
