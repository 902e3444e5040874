// Per-step diagnostics (row A9 of the step): per scene, from the state and
// the fields of the most recent step, the fluid particle count, mean and
// largest neighbour count, the fullest cell of the step's binning, the
// fluid momentum and kinetic energy, the density range and mean, and the
// largest fluid speed.  Two launches, both deterministic and graph-safe:
// blocks of 8,192 slots (and cells) write float64 partials, reduced in a
// fixed tree; then one block per scene adds its partials in chunk order.
#include "sph_internal.cuh"

namespace sphk {

namespace {
constexpr int ST_THREADS = 256;
// partial fields
enum { P_FLUID, P_NBR_SUM, P_NBR_MAX, P_CELL_MAX, P_MX, P_MY, P_MZ, P_V2, P_RHO_MIN, P_RHO_MAX, P_RHO_SUM,
       P_SPEED_MAX, P_N };
static_assert(P_N == STATS_PART, "partial layout");
static_assert(STATS_OUT == SPH_STATS_N, "output layout");

__device__ __forceinline__ bool is_max_field(int f)
{
    return f == P_NBR_MAX || f == P_CELL_MAX || f == P_RHO_MAX || f == P_SPEED_MAX;
}

// v = combine(v, w) field by field (sums, maxima, the minimum)
__device__ __forceinline__ void combine(double* v, const double* w)
{
#pragma unroll
    for (int f = 0; f < P_N; ++f) {
        if (f == P_RHO_MIN) v[f] = fmin(v[f], w[f]);
        else if (is_max_field(f)) v[f] = fmax(v[f], w[f]);
        else v[f] += w[f];
    }
}
}  // namespace

__global__ void __launch_bounds__(ST_THREADS)
k_stats_partial(const float4* __restrict__ pos, const float4* __restrict__ vel, const float* __restrict__ rho,
                const int* __restrict__ nbr, const unsigned* __restrict__ cell_start, Scenes sc, int chunks,
                double* __restrict__ part)
{
    __shared__ double red[ST_THREADS / 32][P_N];
    const int k = blockIdx.y, ch = blockIdx.x, t = threadIdx.x;
    const unsigned p0 = sc.pbase[k], p1 = sc.pbase[k + 1];
    const int ncell = sc.c[k].g.ncells, cbase = sc.c[k].c_base;
    const unsigned nb_all = (unsigned)sc.nb_all;
    double v[P_N];
#pragma unroll
    for (int f = 0; f < P_N; ++f) v[f] = 0.0;
    v[P_RHO_MIN] = INFINITY;
    v[P_RHO_MAX] = -INFINITY;
    const unsigned lo = p0 + (unsigned)ch * STATS_CHUNK;
    const unsigned hi = lo + STATS_CHUNK < p1 ? lo + STATS_CHUNK : p1;
    for (unsigned i = lo + t; i < hi; i += ST_THREADS) {
        const unsigned id = __float_as_uint(pos[i].w);
        if (id < nb_all) continue;  // a boid-attached particle
        const float4 u = vel[i];
        const double ux = u.x, uy = u.y, uz = u.z;
        const double v2 = ux * ux + uy * uy + uz * uz;
        const double r = rho[i];
        v[P_FLUID] += 1.0;
        v[P_NBR_SUM] += (double)nbr[i];
        v[P_NBR_MAX] = fmax(v[P_NBR_MAX], (double)nbr[i]);
        v[P_MX] += ux;
        v[P_MY] += uy;
        v[P_MZ] += uz;
        v[P_V2] += v2;
        v[P_RHO_MIN] = fmin(v[P_RHO_MIN], r);
        v[P_RHO_MAX] = fmax(v[P_RHO_MAX], r);
        v[P_RHO_SUM] += r;
        v[P_SPEED_MAX] = fmax(v[P_SPEED_MAX], sqrt(v2));
    }
    const int c_lo = ch * STATS_CHUNK;
    const int c_hi = c_lo + STATS_CHUNK < ncell ? c_lo + STATS_CHUNK : ncell;
    for (int c = c_lo + t; c < c_hi; c += ST_THREADS)
        v[P_CELL_MAX] = fmax(v[P_CELL_MAX], (double)(cell_start[cbase + c + 1] - cell_start[cbase + c]));
    // fixed-order tree: lanes by xor shuffles, then the warps in order
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        double w[P_N];
#pragma unroll
        for (int f = 0; f < P_N; ++f) w[f] = __shfl_xor_sync(0xffffffffu, v[f], off);
        combine(v, w);
    }
    if ((t & 31) == 0)
#pragma unroll
        for (int f = 0; f < P_N; ++f) red[t >> 5][f] = v[f];
    __syncthreads();
    if (t < P_N) {
        const int f = t;
        double a = red[0][f];
        for (int w = 1; w < ST_THREADS / 32; ++w) {
            const double b = red[w][f];
            a = f == P_RHO_MIN ? fmin(a, b) : is_max_field(f) ? fmax(a, b) : a + b;
        }
        part[((size_t)k * chunks + ch) * P_N + f] = a;
    }
}

// One block per scene: its chunks' partials in order, then the statistics.
__global__ void k_stats_final(const double* __restrict__ part, int chunks, Scenes sc, double* __restrict__ out)
{
    const int k = blockIdx.x, f = threadIdx.x;
    __shared__ double tot[P_N];
    if (f < P_N) {
        double a = part[(size_t)k * chunks * P_N + f];
        for (int c = 1; c < chunks; ++c) {
            const double b = part[((size_t)k * chunks + c) * P_N + f];
            a = f == P_RHO_MIN ? fmin(a, b) : is_max_field(f) ? fmax(a, b) : a + b;
        }
        tot[f] = a;
    }
    __syncthreads();
    if (f == 0) {
        const double m = sc.c[k].mass, nf = tot[P_FLUID];
        double* o = out + (size_t)k * STATS_OUT;
        o[0] = nf;
        o[1] = nf > 0 ? tot[P_NBR_SUM] / nf : 0.0;
        o[2] = tot[P_NBR_MAX];
        o[3] = tot[P_CELL_MAX];
        o[4] = m * tot[P_MX];
        o[5] = m * tot[P_MY];
        o[6] = m * tot[P_MZ];
        o[7] = 0.5 * m * tot[P_V2];
        o[8] = nf > 0 ? tot[P_RHO_MIN] : 0.0;
        o[9] = nf > 0 ? tot[P_RHO_MAX] : 0.0;
        o[10] = nf > 0 ? tot[P_RHO_SUM] / nf : 0.0;
        o[11] = tot[P_SPEED_MAX];
    }
}

cudaError_t launch_stats(const float4* pos, const float4* vel, const float* rho, const int* nbr,
                         const unsigned* cell_start, const Scenes& sc, int chunks, double* part, double* out,
                         cudaStream_t s, long long* launches)
{
    k_stats_partial<<<dim3((unsigned)chunks, (unsigned)sc.S), ST_THREADS, 0, s>>>(pos, vel, rho, nbr, cell_start,
                                                                                   sc, chunks, part);
    k_stats_final<<<sc.S, 32, 0, s>>>(part, chunks, sc, out);
    *launches += 2;
    return cudaGetLastError();
}

}  // namespace sphk
