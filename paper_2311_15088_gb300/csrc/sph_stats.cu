// Per-step diagnostics (row A9 of the step): per scene, from the state and
// the fields of the most recent step, the fluid particle count, mean and
// largest neighbour count, the fullest cell of the step's binning, the
// fluid momentum and kinetic energy, the density range and mean, and the
// largest fluid speed.  Two launches, both deterministic and graph-safe:
// blocks of 2,048 slots (and cells) reduce in a fixed tree (per thread in
// float32 over its 8 slots, then counts as integers, extrema as float32 and
// the sums in float64) and write float64 partials; then one block per scene
// adds its partials, each thread a fixed strided subset, then a fixed tree.
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

// One block's running values, typed so that only the five true sums take
// the float64 pipe: counts and the neighbour sum as integers, extrema as
// float32 (both exact), momentum, |v|^2 and density sums in float64 (each
// thread first sums its at most STATS_CHUNK / ST_THREADS slots in float32).
struct BlockAcc {
    int fluid, nbr_max, cell_max;
    long long nbr_sum;
    double mx, my, mz, v2, rho_sum;
    float rho_min, rho_max, speed_max;
};

__device__ __forceinline__ void acc_combine(BlockAcc& a, const BlockAcc& b)
{
    a.fluid += b.fluid;
    a.nbr_max = max(a.nbr_max, b.nbr_max);
    a.cell_max = max(a.cell_max, b.cell_max);
    a.nbr_sum += b.nbr_sum;
    a.mx += b.mx;
    a.my += b.my;
    a.mz += b.mz;
    a.v2 += b.v2;
    a.rho_sum += b.rho_sum;
    a.rho_min = fminf(a.rho_min, b.rho_min);
    a.rho_max = fmaxf(a.rho_max, b.rho_max);
    a.speed_max = fmaxf(a.speed_max, b.speed_max);
}

__device__ __forceinline__ BlockAcc acc_shfl(const BlockAcc& a, int off)
{
    BlockAcc b;
    b.fluid = __shfl_xor_sync(0xffffffffu, a.fluid, off);
    b.nbr_max = __shfl_xor_sync(0xffffffffu, a.nbr_max, off);
    b.cell_max = __shfl_xor_sync(0xffffffffu, a.cell_max, off);
    b.nbr_sum = __shfl_xor_sync(0xffffffffu, a.nbr_sum, off);
    b.mx = __shfl_xor_sync(0xffffffffu, a.mx, off);
    b.my = __shfl_xor_sync(0xffffffffu, a.my, off);
    b.mz = __shfl_xor_sync(0xffffffffu, a.mz, off);
    b.v2 = __shfl_xor_sync(0xffffffffu, a.v2, off);
    b.rho_sum = __shfl_xor_sync(0xffffffffu, a.rho_sum, off);
    b.rho_min = __shfl_xor_sync(0xffffffffu, a.rho_min, off);
    b.rho_max = __shfl_xor_sync(0xffffffffu, a.rho_max, off);
    b.speed_max = __shfl_xor_sync(0xffffffffu, a.speed_max, off);
    return b;
}

// Fixed-order block reduction of the ST_THREADS threads' values (double
// fields, combined as in `combine`): lanes by xor shuffles, then the warps
// in order; the result lands in red[0].
__device__ __forceinline__ void block_reduce(double (&v)[P_N], double (&red)[ST_THREADS / 32][P_N])
{
    const int t = threadIdx.x;
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
        red[0][f] = a;
    }
    __syncthreads();
}

__device__ __forceinline__ void identity(double (&v)[P_N])
{
#pragma unroll
    for (int f = 0; f < P_N; ++f) v[f] = 0.0;
    v[P_RHO_MIN] = INFINITY;
    v[P_RHO_MAX] = -INFINITY;
}

__global__ void __launch_bounds__(ST_THREADS)
k_stats_partial(const float4* __restrict__ pos, const float4* __restrict__ vel, const float* __restrict__ rho,
                const int* __restrict__ nbr, const unsigned* __restrict__ cell_start, Scenes sc, int chunks,
                double* __restrict__ part)
{
    __shared__ BlockAcc red[ST_THREADS / 32];
    const int k = blockIdx.y, ch = blockIdx.x, t = threadIdx.x;
    const unsigned p0 = sc.pbase[k], p1 = sc.pbase[k + 1];
    const int ncell = sc.c[k].g.ncells, cbase = sc.c[k].c_base;
    const unsigned nb_all = (unsigned)sc.nb_all;
    int fluid = 0, nbr_max = 0, cell_max = 0, nbr_sum = 0;
    float mx = 0.f, my = 0.f, mz = 0.f, v2s = 0.f, rs = 0.f;
    float rho_min = INFINITY, rho_max = -INFINITY, vmax = 0.f;
    const unsigned lo = p0 + (unsigned)ch * STATS_CHUNK;
    const unsigned hi = lo + STATS_CHUNK < p1 ? lo + STATS_CHUNK : p1;
    for (unsigned i = lo + t; i < hi; i += ST_THREADS) {
        const unsigned id = __float_as_uint(pos[i].w);
        if (id < nb_all) continue;  // a boid-attached particle
        const float4 u = vel[i];
        const float v2 = fmaf(u.z, u.z, fmaf(u.y, u.y, u.x * u.x));
        const float r = rho[i];
        const int nn = nbr[i];
        ++fluid;
        nbr_sum += nn;
        nbr_max = max(nbr_max, nn);
        mx += u.x;
        my += u.y;
        mz += u.z;
        v2s += v2;
        rs += r;
        rho_min = fminf(rho_min, r);
        rho_max = fmaxf(rho_max, r);
        vmax = fmaxf(vmax, sqrtf(v2));
    }
    const int c_lo = ch * STATS_CHUNK;
    const int c_hi = c_lo + STATS_CHUNK < ncell ? c_lo + STATS_CHUNK : ncell;
    for (int c = c_lo + t; c < c_hi; c += ST_THREADS)
        cell_max = max(cell_max, (int)(cell_start[cbase + c + 1] - cell_start[cbase + c]));
    BlockAcc a{fluid, nbr_max, cell_max, (long long)nbr_sum, (double)mx, (double)my, (double)mz, (double)v2s,
               (double)rs, rho_min, rho_max, vmax};
    // fixed-order tree: lanes by xor shuffles, then the warps in order
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc_combine(a, acc_shfl(a, off));
    if ((t & 31) == 0) red[t >> 5] = a;
    __syncthreads();
    if (t == 0) {
        BlockAcc b = red[0];
        for (int w = 1; w < ST_THREADS / 32; ++w) acc_combine(b, red[w]);
        double* o = part + ((size_t)k * chunks + ch) * P_N;
        o[P_FLUID] = (double)b.fluid;
        o[P_NBR_SUM] = (double)b.nbr_sum;
        o[P_NBR_MAX] = (double)b.nbr_max;
        o[P_CELL_MAX] = (double)b.cell_max;
        o[P_MX] = b.mx;
        o[P_MY] = b.my;
        o[P_MZ] = b.mz;
        o[P_V2] = b.v2;
        o[P_RHO_MIN] = (double)b.rho_min;
        o[P_RHO_MAX] = (double)b.rho_max;
        o[P_RHO_SUM] = b.rho_sum;
        o[P_SPEED_MAX] = (double)b.speed_max;
    }
}

// One block per scene: thread t combines chunks t, t + ST_THREADS, ... in
// order (chunks past the scene's own hold identities, which change no bit),
// then the block tree; then the statistics.
__global__ void __launch_bounds__(ST_THREADS)
k_stats_final(const double* __restrict__ part, int chunks, Scenes sc, double* __restrict__ out)
{
    __shared__ double red[ST_THREADS / 32][P_N];
    const int k = blockIdx.x, t = threadIdx.x;
    double v[P_N];
    identity(v);
    for (int c = t; c < chunks; c += ST_THREADS) {
        double w[P_N];
#pragma unroll
        for (int f = 0; f < P_N; ++f) w[f] = part[((size_t)k * chunks + c) * P_N + f];
        combine(v, w);
    }
    block_reduce(v, red);
    if (t == 0) {
        const double* tot = red[0];
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
    k_stats_final<<<sc.S, ST_THREADS, 0, s>>>(part, chunks, sc, out);
    *launches += 2;
    return cudaGetLastError();
}

}  // namespace sphk
