// sph_surface.cu -- surface reconstruction from the particles: the voxel
// density on a grid of corners (section "Voxel Density") and marching cubes
// into a triangle buffer in device memory (section "Marching Cubes").
//
// Voxel density at corner x: phi(x) = |x - xbar| - r with
// xbar = sum_i w_i x_i, w_i = k(|x - x_i| / R) / sum_j k(|x - x_j| / R),
// k(s) = (1 - s^2)^3, over the fluid particles with |x - x_i| < R (the
// float32 predicate of the step's neighbour search with R for h).  Evaluated
// as phi = |sum_i k_i (x_i - x)| / sum_i k_i - r: the same value, with the
// offsets x_i - x (already formed for the predicate) instead of absolute
// positions, so float32 loses nothing to the size of the coordinates.  A
// corner without neighbours gets phi = R.  One thread per corner, walking
// the rows of the particle grid that its R-sphere can reach (RowWalk), in
// slot order.
//
// Marching cubes: cube (ix, iy, iz) has vertex v at corner (ix, iy, iz) +
// (0,0,0), (1,0,0), (1,1,0), (0,1,0), (0,0,1), (1,0,1), (1,1,1), (0,1,1)
// for v = 0 .. 7 and edges (v0 v1), (v1 v2), (v2 v3), (v3 v0), (v4 v5),
// (v5 v6), (v6 v7), (v7 v4), (v0 v4), (v1 v5), (v2 v6), (v3 v7) -- the
// numbering of the paper's worked example (vertex 3 alone below the
// isovalue: cube index 8, edges 2, 3, 11 cut).  Cube index bit v is set when
// the value at vertex v is below the isovalue.  A cut edge's vertex is
// p1 + (iso - v1) / (v2 - v1) (p2 - p1) with p1 the endpoint of smaller
// coordinate, so the cubes sharing an edge compute the same bits.  Three
// passes: count the triangles of every cube, exclusive scan, emit them in
// cube order (each cube's in table order) into the caller's buffer.
//
// The tables are generated on the host at first use (mc_case, below) from
// the cube's numbering and copied to each device before the first
// marching-cubes launch on it: the triangle table and counts go to global
// memory (the threads of a warp index them by different cases, which the
// constant cache would serialise); the edge table stays on the host
// (sph_mc_tables).
#include <math.h>
#include <string.h>

#include <mutex>

#include "sph_internal.cuh"

namespace sphk {

__device__ signed char c_mc_tri[256][16];
__device__ unsigned char c_mc_ntri[256];

// ------------------------------------------------------ table generation

namespace {
const int V[8][3] = {{0, 0, 0}, {1, 0, 0}, {1, 1, 0}, {0, 1, 0}, {0, 0, 1}, {1, 0, 1}, {1, 1, 1}, {0, 1, 1}};
const int E[12][2] = {{0, 1}, {1, 2}, {2, 3}, {3, 0}, {4, 5}, {5, 6}, {6, 7}, {7, 4}, {0, 4}, {1, 5}, {2, 6}, {3, 7}};
// faces as vertex cycles and their outward normals
const int F[6][4] = {{0, 1, 2, 3}, {4, 5, 6, 7}, {0, 1, 5, 4}, {1, 2, 6, 5}, {2, 3, 7, 6}, {3, 0, 4, 7}};
const int FN[6][3] = {{0, 0, -1}, {0, 0, 1}, {0, -1, 0}, {1, 0, 0}, {0, 1, 0}, {-1, 0, 0}};

int edge_between(int a, int b)
{
    for (int e = 0; e < 12; ++e)
        if ((E[e][0] == a && E[e][1] == b) || (E[e][0] == b && E[e][1] == a)) return e;
    return -1;
}

// faces containing edge e, as a bit mask
int faces_of(int e)
{
    int m = 0;
    for (int f = 0; f < 6; ++f) {
        bool u = false, v = false;
        for (int k = 0; k < 4; ++k) {
            u |= F[f][k] == E[e][0];
            v |= F[f][k] == E[e][1];
        }
        if (u && v) m |= 1 << f;
    }
    return m;
}

void midpoint(int e, double m[3])
{
    for (int a = 0; a < 3; ++a) m[a] = 0.5 * (V[E[e][0]][a] + V[E[e][1]][a]);
}

// One case: every face adds the segments that cut its corners below the
// isovalue off -- between its two cut edges, or, with four cut edges, one
// around each of its two corners below (a rule of the face alone, so the
// neighbouring cube agrees) -- directed so that (outward normal) x
// (direction) points at the corners cut off; the segments chain into closed
// loops; each loop (in order of its smallest edge) is fanned into triangles
// from its smallest edge, or from the next edge along it whose fan puts no
// triangle in a cube face.  Returns the number of triangles (<= 5), or -1.
int mc_case(int ci, unsigned short* edge_mask, signed char tri[16])
{
    bool in[8];
    for (int v = 0; v < 8; ++v) in[v] = (ci >> v) & 1;
    unsigned short mask = 0;
    for (int e = 0; e < 12; ++e)
        if (in[E[e][0]] != in[E[e][1]]) mask |= (unsigned short)(1u << e);
    *edge_mask = mask;
    int nxt[12];
    for (int e = 0; e < 12; ++e) nxt[e] = -1;
    for (int f = 0; f < 6; ++f) {
        int seg_a[2], seg_b[2], seg_c[2][4], seg_nc[2], nseg = 0;
        int cut[4], ncut = 0;
        for (int k = 0; k < 4; ++k)
            if (in[F[f][k]] != in[F[f][(k + 1) % 4]]) cut[ncut++] = edge_between(F[f][k], F[f][(k + 1) % 4]);
        if (ncut == 2) {
            seg_a[0] = cut[0];
            seg_b[0] = cut[1];
            seg_nc[0] = 0;
            for (int k = 0; k < 4; ++k)
                if (in[F[f][k]]) seg_c[0][seg_nc[0]++] = F[f][k];
            nseg = 1;
        } else if (ncut == 4) {
            for (int k = 0; k < 4; ++k)
                if (in[F[f][k]]) {
                    seg_a[nseg] = edge_between(F[f][(k + 3) % 4], F[f][k]);
                    seg_b[nseg] = edge_between(F[f][k], F[f][(k + 1) % 4]);
                    seg_c[nseg][0] = F[f][k];
                    seg_nc[nseg] = 1;
                    ++nseg;
                }
        } else if (ncut != 0) {
            return -1;
        }
        for (int s = 0; s < nseg; ++s) {
            double ma[3], mb[3], t[3], side[3], cr[3];
            midpoint(seg_a[s], ma);
            midpoint(seg_b[s], mb);
            for (int a = 0; a < 3; ++a) {
                t[a] = mb[a] - ma[a];
                double c = 0.0;
                for (int k = 0; k < seg_nc[s]; ++k) c += V[seg_c[s][k]][a];
                side[a] = c / seg_nc[s] - 0.5 * (ma[a] + mb[a]);
            }
            cr[0] = FN[f][1] * t[2] - FN[f][2] * t[1];
            cr[1] = FN[f][2] * t[0] - FN[f][0] * t[2];
            cr[2] = FN[f][0] * t[1] - FN[f][1] * t[0];
            int a = seg_a[s], b = seg_b[s];
            if (cr[0] * side[0] + cr[1] * side[1] + cr[2] * side[2] < 0.0) {
                const int tmp = a;
                a = b;
                b = tmp;
            }
            if (nxt[a] != -1) return -1;
            nxt[a] = b;
        }
    }
    int ntri = 0;
    bool used[12] = {false};
    for (;;) {
        int e0 = -1;
        for (int e = 0; e < 12; ++e)
            if (nxt[e] != -1 && !used[e]) {
                e0 = e;
                break;
            }
        if (e0 < 0) break;
        int loop[12], L = 0;
        for (int e = e0; L == 0 || e != e0; e = nxt[e]) {
            if (L == 12 || nxt[e] == -1) return -1;
            loop[L++] = e;
            used[e] = true;
        }
        int start = -1;
        for (int r = 0; r < L && start < 0; ++r) {
            bool ok = true;
            for (int i = 1; i + 1 < L; ++i) {
                const int x = loop[r], y = loop[(r + i) % L], z = loop[(r + i + 1) % L];
                if (faces_of(x) & faces_of(y) & faces_of(z)) ok = false;
            }
            if (ok) start = r;
        }
        if (start < 0) return -1;
        for (int i = 1; i + 1 < L; ++i) {
            if (ntri == 5) return -1;
            tri[3 * ntri] = (signed char)loop[start];
            tri[3 * ntri + 1] = (signed char)loop[(start + i) % L];
            tri[3 * ntri + 2] = (signed char)loop[(start + i + 1) % L];
            ++ntri;
        }
    }
    for (int k = 3 * ntri; k < 16; ++k) tri[k] = -1;
    for (int e = 0; e < 12; ++e)
        if (((mask >> e) & 1) != (nxt[e] != -1)) return -1;
    return ntri;
}

struct McTables {
    unsigned short edge[256];
    signed char tri[256][16];
    unsigned char ntri[256];
    int ok;
};

const McTables& host_tables()
{
    static McTables t;
    static std::once_flag once;
    std::call_once(once, [] {
        t.ok = 1;
        for (int ci = 0; ci < 256; ++ci) {
            const int n = mc_case(ci, &t.edge[ci], t.tri[ci]);
            if (n < 0) {
                t.ok = 0;
                t.ntri[ci] = 0;
                continue;
            }
            t.ntri[ci] = (unsigned char)n;
        }
    });
    return t;
}

// The device whose constant memory holds the tables (one flag per device).
constexpr int MAX_DEVICES = 64;
bool g_uploaded[MAX_DEVICES];
std::mutex g_upload_mutex;
}  // namespace

int mc_tables_host(unsigned short* edge, signed char* tri)
{
    const McTables& t = host_tables();
    if (!t.ok) return -1;
    if (edge) memcpy(edge, t.edge, sizeof(t.edge));
    if (tri) memcpy(tri, t.tri, sizeof(t.tri));
    return 0;
}

cudaError_t mc_upload_tables()
{
    const McTables& t = host_tables();
    if (!t.ok) return cudaErrorInvalidValue;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_upload_mutex);
    if (g_uploaded[dev]) return cudaSuccess;
    e = cudaMemcpyToSymbol(c_mc_tri, t.tri, sizeof(t.tri));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_mc_ntri, t.ntri, sizeof(t.ntri));
    if (e == cudaSuccess) g_uploaded[dev] = true;
    return e;
}

// --------------------------------------------------------- voxel density

__global__ void __launch_bounds__(256)
k_voxel_density(const float4* __restrict__ pos, const unsigned* __restrict__ start, Scenes sc, VoxelConst v,
                float* __restrict__ phi, int* __restrict__ count)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long n = (long long)v.dims[0] * v.dims[1] * v.dims[2];
    if (idx >= n) return;
    const int ix = (int)(idx % v.dims[0]);
    const int iy = (int)((idx / v.dims[0]) % v.dims[1]);
    const int iz = (int)(idx / ((long long)v.dims[0] * v.dims[1]));
    const float x = __fadd_rn(__fmul_rn((float)ix, v.spacing), v.origin[0]);
    const float y = __fadd_rn(__fmul_rn((float)iy, v.spacing), v.origin[1]);
    const float z = __fadd_rn(__fmul_rn((float)iz, v.spacing), v.origin[2]);
    const StepConst& c = sc.c[0];
    const int nb_all = sc.nb_all;
    float ks = 0.0f, kx = 0.0f, ky = 0.0f, kz = 0.0f;
    int cnt = 0;
    RowWalk walk(c.g, v.wb, start + c.c_base, x, y, z);
    unsigned s0, s1;
    while (walk.next(s0, s1)) {
        for (unsigned j = s0; j < s1; ++j) {
            const float4 pj = __ldg(pos + j);
            const float dx = __fsub_rn(pj.x, x), dy = __fsub_rn(pj.y, y), dz = __fsub_rn(pj.z, z);
            const float r2 = pair_r2(dx, dy, dz);
            if (r2 < v.R2 && id_of(pj) >= nb_all) {
                const float t = 1.0f - r2 * v.invR2;
                const float k = t * t * t;
                ks += k;
                kx = fmaf(k, dx, kx);
                ky = fmaf(k, dy, ky);
                kz = fmaf(k, dz, kz);
                ++cnt;
            }
        }
    }
    float f = v.R;
    if (cnt > 0) f = sqrtf(kx * kx + ky * ky + kz * kz) / ks - v.r;
    phi[idx] = f;
    if (count) count[idx] = cnt;
}

cudaError_t launch_voxel_density(const float4* pos, const unsigned* start, const Scenes& sc, const VoxelConst& v,
                                 float* phi, int* count, cudaStream_t s, long long* launches)
{
    const long long n = (long long)v.dims[0] * v.dims[1] * v.dims[2];
    if (n <= 0) return cudaSuccess;
    k_voxel_density<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(pos, start, sc, v, phi, count);
    ++*launches;
    return cudaGetLastError();
}

// -------------------------------------------------------- marching cubes

struct McGrid {
    int nx, ny, nz;      // corners per axis
    float origin[3], spacing, iso;
};

// Index of corner (ix, iy, iz) and coordinates of cube c, in 32-bit
// arithmetic: a corner grid holds fewer than 2^31 corners (checked before
// any launch).
__device__ __forceinline__ unsigned mc_corner(const McGrid& g, int ix, int iy, int iz)
{
    return (unsigned)ix + (unsigned)g.nx * ((unsigned)iy + (unsigned)g.ny * (unsigned)iz);
}

__device__ __forceinline__ void mc_cube_coords(const McGrid& g, unsigned c, int ii[3])
{
    const unsigned cx = (unsigned)(g.nx - 1), cy = (unsigned)(g.ny - 1);
    const unsigned r = c / cx, z = r / cy;
    ii[0] = (int)(c - r * cx);
    ii[1] = (int)(r - z * cy);
    ii[2] = (int)z;
}

// The values at the eight vertices of cube ii, and the cube's case.
__device__ __forceinline__ void cube_values(const float* __restrict__ phi, const McGrid& g, const int ii[3],
                                            float val[8])
{
#pragma unroll
    for (int v = 0; v < 8; ++v) {
        const int ox = (v == 1 || v == 2 || v == 5 || v == 6), oy = (v == 2 || v == 3 || v == 6 || v == 7),
                  oz = v >= 4;
        val[v] = __ldg(phi + mc_corner(g, ii[0] + ox, ii[1] + oy, ii[2] + oz));
    }
}

__device__ __forceinline__ int cube_case(const McGrid& g, const float val[8])
{
    int ci = 0;
#pragma unroll
    for (int v = 0; v < 8; ++v) ci |= (val[v] < g.iso) << v;
    return ci;
}

// Edge endpoints, the one of smaller coordinate first, and the vertex
// offsets (bit 0: +x, bit 1: +y, bit 2: +z) of the numbering above, packed
// three bits per entry so that a lookup is a shift (entry k of a table:
// (bits >> 3 k) & 7), with no memory access.
constexpr unsigned char MC_LO[12] = {0, 1, 3, 0, 4, 5, 7, 4, 0, 1, 2, 3};
constexpr unsigned char MC_HI[12] = {1, 2, 2, 3, 5, 6, 6, 7, 4, 5, 6, 7};
constexpr unsigned char MC_OFF[8] = {0, 1, 3, 2, 4, 5, 7, 6};

template <int N>
constexpr unsigned long long mc_pack3(const unsigned char (&t)[N])
{
    unsigned long long b = 0;
    for (int k = 0; k < N; ++k) b |= (unsigned long long)t[k] << (3 * k);
    return b;
}
constexpr unsigned long long MC_LO3 = mc_pack3(MC_LO), MC_HI3 = mc_pack3(MC_HI), MC_OFF3 = mc_pack3(MC_OFF);

// Triangle k of cube ii (case ci), written to out[0 .. 9); each vertex
// reads its edge's two corner values from phi.
__device__ __forceinline__ void mc_emit_tri(const float* __restrict__ phi, const McGrid& g, const int ii[3], int ci,
                                            int k, float* __restrict__ out)
{
    // corner of offset bits b (bit 0: +x, bit 1: +y, bit 2: +z)
    auto corner = [&](int b) {
        return __ldg(phi + mc_corner(g, ii[0] + (b & 1), ii[1] + ((b >> 1) & 1), ii[2] + (b >> 2)));
    };
    float lo[3], hi[3];  // the cube's corner coordinates, fl(origin + fl(i * spacing))
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        lo[a] = __fadd_rn(__fmul_rn((float)ii[a], g.spacing), g.origin[a]);
        hi[a] = __fadd_rn(__fmul_rn((float)(ii[a] + 1), g.spacing), g.origin[a]);
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const int e = __ldg(&c_mc_tri[ci][3 * k + q]);
        const int v1 = (int)(MC_LO3 >> (3 * e)) & 7, v2 = (int)(MC_HI3 >> (3 * e)) & 7;
        const int b1 = (int)(MC_OFF3 >> (3 * v1)) & 7, b2 = (int)(MC_OFF3 >> (3 * v2)) & 7;
        const float f1 = corner(b1), f2 = corner(b2);
        const float t = __fdiv_rn(__fsub_rn(g.iso, f1), __fsub_rn(f2, f1));
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float p1 = (b1 >> a) & 1 ? hi[a] : lo[a];
            const float p2 = (b2 >> a) & 1 ? hi[a] : lo[a];
            out[3 * q + a] = __fadd_rn(p1, __fmul_rn(t, __fsub_rn(p2, p1)));
        }
    }
}

// Marching cubes in three launches, without a wait between blocks, over
// tiles of MC_TILE consecutive cubes (MC_CPT per thread of an MC_T-thread
// block).  k_mc_tile_counts (a block per tile) stores every cube's case
// byte and the tile's triangle total; k_mc_tile_scan (one block) turns the
// totals into the tiles' offsets and the grand total; k_mc_tile_emit
// (MC_SPLIT blocks per tile with triangles) scans the tile's counts in
// shared memory in each block and then spreads the tile's triangles evenly
// over the threads of its blocks: triangle q
// of the tile belongs to the cube u with pre[u] <= q < pre[u + 1] (a binary
// search of the scan), and a warp's 32 consecutive triangles go out through
// shared memory as one contiguous run.  The output is in cube order, as if
// the counts had been scanned over the whole grid.
constexpr int MC_T = 256, MC_CPT = 4, MC_TILE = MC_T * MC_CPT;
// emit blocks per tile (blockIdx.y); block y takes the runs of MC_T triangles y, y + MC_SPLIT, ...
constexpr int MC_SPLIT = 4;

// Exclusive prefix of v over the block (MC_T threads) and the block total.
__device__ __forceinline__ unsigned mc_block_scan(unsigned v, unsigned* s_warp, unsigned& total)
{
    const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    unsigned inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned u = __shfl_up_sync(FULL, inc, o);
        if (lane >= (unsigned)o) inc += u;
    }
    if (lane == 31u) s_warp[warp] = inc;
    __syncthreads();
    unsigned before = 0, all = 0;
#pragma unroll
    for (int w = 0; w < MC_T / 32; ++w) {
        const unsigned t = s_warp[w];
        before += (unsigned)w < warp ? t : 0u;
        all += t;
    }
    total = all;
    return before + inc - v;
}

// Thread t takes cubes c0 + t + k MC_T (k < MC_CPT): all their corner loads
// first (a thread past the end loads cube 0's), then their cases.
__global__ void __launch_bounds__(MC_T)
k_mc_tile_counts(const float* __restrict__ phi, McGrid g, unsigned char* __restrict__ cases,
                 unsigned* __restrict__ tile_count)
{
    __shared__ unsigned s_sum[MC_T / 32];
    const unsigned n = (unsigned)(g.nx - 1) * (unsigned)(g.ny - 1) * (unsigned)(g.nz - 1);
    const unsigned c0 = blockIdx.x * MC_TILE + threadIdx.x;
    float val[MC_CPT][8];
#pragma unroll
    for (int k = 0; k < MC_CPT; ++k) {
        const unsigned c = c0 + k * MC_T;
        int ii[3];
        mc_cube_coords(g, c < n ? c : 0u, ii);
        cube_values(phi, g, ii, val[k]);
    }
    unsigned mine = 0;
#pragma unroll
    for (int k = 0; k < MC_CPT; ++k) {
        const unsigned c = c0 + k * MC_T;
        if (c < n) {
            const int ci = cube_case(g, val[k]);
            cases[c] = (unsigned char)ci;
            mine += __ldg(c_mc_ntri + ci);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(FULL, mine, o);
    if ((threadIdx.x & 31u) == 0) s_sum[threadIdx.x >> 5] = mine;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned tot = 0;
#pragma unroll
        for (int w = 0; w < MC_T / 32; ++w) tot += s_sum[w];
        tile_count[blockIdx.x] = tot;
    }
}

// One block of 1024 threads: thread t sums its run of consecutive tile
// totals, the block scans those sums, and the thread writes its tiles'
// offsets (64-bit); the grand total, saturated to 0xfffffffe, goes to
// *total_out.
__global__ void __launch_bounds__(1024)
k_mc_tile_scan(const unsigned* __restrict__ tile_count, int ntiles, unsigned long long* __restrict__ tile_off,
               unsigned* __restrict__ total_out)
{
    __shared__ unsigned long long s_warp[32];
    const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const int per = (ntiles + 1023) / 1024;
    const int a = (int)threadIdx.x * per, e = min(a + per, ntiles);
    unsigned long long mine = 0;
    for (int t0 = a; t0 < e; t0 += 8) {  // eight loads in flight
        unsigned x[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) x[j] = t0 + j < e ? __ldg(tile_count + t0 + j) : 0u;
#pragma unroll
        for (int j = 0; j < 8; ++j) mine += x[j];
    }
    unsigned long long inc = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long u = __shfl_up_sync(FULL, inc, o);
        if (lane >= (unsigned)o) inc += u;
    }
    if (lane == 31u) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        unsigned long long x = s_warp[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long u = __shfl_up_sync(FULL, x, o);
            if (lane >= (unsigned)o) x += u;
        }
        s_warp[lane] = x;  // inclusive over the warps
    }
    __syncthreads();
    unsigned long long run = (warp ? s_warp[warp - 1] : 0ull) + inc - mine;
    for (int t = a; t < e; ++t) {
        tile_off[t] = run;
        run += __ldg(tile_count + t);
    }
    if (threadIdx.x == 1023) {
        const unsigned long long tot = s_warp[31];
        *total_out = tot > 0xfffffffeull ? 0xfffffffeu : (unsigned)tot;
    }
}

__global__ void __launch_bounds__(MC_T)
k_mc_tile_emit(const float* __restrict__ phi, McGrid g, const unsigned char* __restrict__ cases,
               const unsigned* __restrict__ tile_count, const unsigned long long* __restrict__ tile_off,
               float* __restrict__ tris, unsigned long long cap)
{
    if (__ldg(tile_count + blockIdx.x) == 0) return;  // a tile without triangles (uniform)
    __shared__ unsigned s_warp[MC_T / 32];
    __shared__ unsigned s_pre[MC_TILE + 1];
    __shared__ unsigned char s_case[MC_TILE];
    __shared__ float s_out[MC_T / 32][32 * 9];
    const unsigned n = (unsigned)(g.nx - 1) * (unsigned)(g.ny - 1) * (unsigned)(g.nz - 1);
    const unsigned c0 = blockIdx.x * MC_TILE;
    // this thread's MC_CPT consecutive cubes: their case bytes in one load
    // (the case array is padded to 256 bytes), those past the end as case 0
    const unsigned cb = c0 + MC_CPT * threadIdx.x;
    static_assert(MC_CPT == 4, "one 4-byte load of case bytes");
    const uchar4 q4 = cb < n ? __ldg(reinterpret_cast<const uchar4*>(cases + cb)) : make_uchar4(0, 0, 0, 0);
    const int cc[MC_CPT] = {q4.x, q4.y, q4.z, q4.w};
    unsigned pre[MC_CPT], local = 0;
#pragma unroll
    for (int k = 0; k < MC_CPT; ++k) {
        const int ci = cb + k < n ? cc[k] : 0;
        s_case[MC_CPT * threadIdx.x + k] = (unsigned char)ci;
        pre[k] = local;
        local += __ldg(c_mc_ntri + ci);
    }
    unsigned total;
    const unsigned excl = mc_block_scan(local, s_warp, total);
#pragma unroll
    for (int k = 0; k < MC_CPT; ++k) s_pre[MC_CPT * threadIdx.x + k] = excl + pre[k];
    if (threadIdx.x == 0) s_pre[MC_TILE] = total;
    __syncthreads();
    const unsigned long long base = tile_off[blockIdx.x];
    if (base >= cap) return;
    const unsigned lim = cap - base < (unsigned long long)total ? (unsigned)(cap - base) : total;
    const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    float* const buf = s_out[warp];
    for (unsigned q0 = blockIdx.y * MC_T + warp * 32u; q0 < lim; q0 += MC_T * MC_SPLIT) {  // warp-uniform
        const unsigned q = q0 + lane;
        if (q < lim) {
            int lo = 0, hi = MC_TILE;  // s_pre[lo] <= q < s_pre[hi]
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (s_pre[mid] <= q) lo = mid;
                else hi = mid;
            }
            int ii[3];
            mc_cube_coords(g, c0 + (unsigned)lo, ii);
            mc_emit_tri(phi, g, ii, s_case[lo], (int)(q - s_pre[lo]), buf + 9 * lane);
        }
        __syncwarp();
        // the warp's triangles q0 .. q0 + m - 1 are one contiguous run
        const unsigned m = min(32u, lim - q0);
        float* __restrict__ dst = tris + 9ull * (base + q0);
        for (unsigned f = lane; f < 9 * m; f += 32) dst[f] = buf[f];
        __syncwarp();
    }
}

long long mc_tiles(long long ncubes) { return (ncubes + MC_TILE - 1) / MC_TILE; }

cudaError_t launch_marching_cubes(const float* phi, const int dims[3], const float origin[3], float spacing,
                                  float iso, unsigned char* cases, unsigned* tile_count,
                                  unsigned long long* tile_off, unsigned* total, float* tris,
                                  unsigned long long cap, cudaStream_t s, long long* launches)
{
    McGrid g;
    g.nx = dims[0];
    g.ny = dims[1];
    g.nz = dims[2];
    for (int a = 0; a < 3; ++a) g.origin[a] = origin[a];
    g.spacing = spacing;
    g.iso = iso;
    const long long n = (long long)(g.nx - 1) * (g.ny - 1) * (g.nz - 1);
    if (n <= 0) return cudaMemsetAsync(total, 0, sizeof(unsigned), s);
    const int nt = (int)mc_tiles(n);
    k_mc_tile_counts<<<(unsigned)nt, MC_T, 0, s>>>(phi, g, cases, tile_count);
    k_mc_tile_scan<<<1, 1024, 0, s>>>(tile_count, nt, tile_off, total);
    k_mc_tile_emit<<<dim3((unsigned)nt, MC_SPLIT), MC_T, 0, s>>>(phi, g, cases, tile_count, tile_off, tris, cap);
    *launches += 3;
    return cudaGetLastError();
}

}  // namespace sphk
