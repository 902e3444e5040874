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
// the cube's numbering and copied to each device's constant memory before
// the first marching-cubes launch on it.
#include <math.h>
#include <string.h>

#include <mutex>

#include "sph_internal.cuh"

namespace sphk {

__constant__ unsigned short c_mc_edge[256];
__constant__ signed char c_mc_tri[256][16];
__constant__ unsigned char c_mc_ntri[256];

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
    e = cudaMemcpyToSymbol(c_mc_edge, t.edge, sizeof(t.edge));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_mc_tri, t.tri, sizeof(t.tri));
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

__device__ __forceinline__ int cube_case(const float* __restrict__ phi, const McGrid& g, int ix, int iy, int iz,
                                         float val[8])
{
    int ci = 0;
#pragma unroll
    for (int v = 0; v < 8; ++v) {
        const int ox = (v == 1 || v == 2 || v == 5 || v == 6), oy = (v == 2 || v == 3 || v == 6 || v == 7),
                  oz = v >= 4;
        val[v] = __ldg(phi + (ix + ox) + (long long)g.nx * ((iy + oy) + (long long)g.ny * (iz + oz)));
        ci |= (val[v] < g.iso) << v;
    }
    return ci;
}

// Edge endpoints, the one of smaller coordinate first, and the vertex
// offsets (bit 0: +x, bit 1: +y, bit 2: +z) of the numbering above.
__constant__ unsigned char c_mc_lo[12] = {0, 1, 3, 0, 4, 5, 7, 4, 0, 1, 2, 3};
__constant__ unsigned char c_mc_hi[12] = {1, 2, 2, 3, 5, 6, 6, 7, 4, 5, 6, 7};
__constant__ unsigned char c_mc_off[8] = {0, 1, 3, 2, 4, 5, 7, 6};

// The triangles of cube c (index ii, case ci, corner values val) from
// output slot o0 on (slots at or past cap are not written).
__device__ __forceinline__ void mc_emit_cube(const McGrid& g, const int ii[3], int ci, const float val[8],
                                             unsigned long long o0, float* __restrict__ tris,
                                             unsigned long long cap)
{
    float lo[3], hi[3];  // the cube's corner coordinates, fl(origin + fl(i * spacing))
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        lo[a] = __fadd_rn(__fmul_rn((float)ii[a], g.spacing), g.origin[a]);
        hi[a] = __fadd_rn(__fmul_rn((float)(ii[a] + 1), g.spacing), g.origin[a]);
    }
    const int nt = c_mc_ntri[ci];
    for (int k = 0; k < nt; ++k) {
        const unsigned long long slot = o0 + (unsigned long long)k;
        if (slot >= cap) return;
        float* out = tris + 9ull * slot;
        for (int q = 0; q < 3; ++q) {
            const int e = c_mc_tri[ci][3 * k + q];
            const int v1 = c_mc_lo[e], v2 = c_mc_hi[e];
            const float f1 = val[v1], f2 = val[v2];
            const float t = __fdiv_rn(__fsub_rn(g.iso, f1), __fsub_rn(f2, f1));
            const int b1 = c_mc_off[v1], b2 = c_mc_off[v2];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const float p1 = (b1 >> a) & 1 ? hi[a] : lo[a];
                const float p2 = (b2 >> a) & 1 ? hi[a] : lo[a];
                out[3 * q + a] = __fadd_rn(p1, __fmul_rn(t, __fsub_rn(p2, p1)));
            }
        }
    }
}

// Marching cubes in three launches, without a wait between blocks: tiles
// of MC_TILE consecutive cubes (a block each) count their triangles and
// store the tile's total; one block scans the tile totals into tile
// offsets (and the grand total); then each tile recounts its cubes, scans
// them within the block and writes its triangles from its tile's offset.
// The output is in cube order, as if the counts had been scanned over the
// whole grid.
constexpr int MC_T = 256, MC_C = 1, MC_TILE = MC_T * MC_C;

// Cases and triangle counts of this thread's cubes c0 .. c0 + MC_C - 1
// (beyond n: none); returns the thread's total and stores each case byte.
__device__ __forceinline__ unsigned mc_thread_cases(const float* __restrict__ phi, const McGrid& g, long long n,
                                                    long long c0, int ci[MC_C], unsigned char* __restrict__ cases)
{
    const int cx = g.nx - 1, cy = g.ny - 1;
    unsigned mine = 0;
#pragma unroll
    for (int k = 0; k < MC_C; ++k) {
        ci[k] = 0;
        const long long c = c0 + k;
        if (c < n) {
            float val[8];
            ci[k] = cube_case(phi, g, (int)(c % cx), (int)((c / cx) % cy), (int)(c / ((long long)cx * cy)), val);
            cases[c] = (unsigned char)ci[k];
            mine += c_mc_ntri[ci[k]];
        }
    }
    return mine;
}

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

__global__ void __launch_bounds__(MC_T)
k_mc_tile_counts(const float* __restrict__ phi, McGrid g, unsigned char* __restrict__ cases,
                 unsigned* __restrict__ tile_count)
{
    __shared__ unsigned s_warp[MC_T / 32];
    const long long n = (long long)(g.nx - 1) * (g.ny - 1) * (g.nz - 1);
    int ci[MC_C];
    const unsigned mine =
        mc_thread_cases(phi, g, n, (long long)blockIdx.x * MC_TILE + (long long)threadIdx.x * MC_C, ci, cases);
    unsigned total;
    mc_block_scan(mine, s_warp, total);
    if (threadIdx.x == 0) tile_count[blockIdx.x] = total;
}

// One block: tile_off[t] = sum of tile_count[0 .. t-1] (64-bit), and the
// grand total (saturated to 0xfffffffe) in *total_out.
__global__ void __launch_bounds__(1024)
k_mc_tile_scan(const unsigned* __restrict__ tile_count, int ntiles, unsigned long long* __restrict__ tile_off,
               unsigned* __restrict__ total_out)
{
    __shared__ unsigned long long s_warp[32];
    __shared__ unsigned long long s_carry;
    const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (int base = 0; base < ntiles; base += 1024) {
        const int t = base + (int)threadIdx.x;
        const unsigned long long v = t < ntiles ? tile_count[t] : 0ull;
        unsigned long long inc = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long u = __shfl_up_sync(FULL, inc, o);
            if (lane >= (unsigned)o) inc += u;
        }
        if (lane == 31u) s_warp[warp] = inc;
        __syncthreads();
        unsigned long long before = 0, all = 0;
        for (int w = 0; w < 32; ++w) {
            const unsigned long long x = s_warp[w];
            before += (unsigned)w < warp ? x : 0ull;
            all += x;
        }
        const unsigned long long carry = s_carry;
        if (t < ntiles) tile_off[t] = carry + before + inc - v;
        __syncthreads();  // every thread has read s_warp and s_carry
        if (threadIdx.x == 0) s_carry = carry + all;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const unsigned long long tot = s_carry;
        *total_out = tot > 0xfffffffeull ? 0xfffffffeu : (unsigned)tot;
    }
}

__global__ void __launch_bounds__(MC_T)
k_mc_tile_emit(const float* __restrict__ phi, McGrid g, const unsigned char* __restrict__ cases,
               const unsigned long long* __restrict__ tile_off, float* __restrict__ tris, unsigned long long cap)
{
    __shared__ unsigned s_warp[MC_T / 32];
    const int cx = g.nx - 1, cy = g.ny - 1;
    const long long n = (long long)cx * cy * (g.nz - 1);
    const long long c0 = (long long)blockIdx.x * MC_TILE + (long long)threadIdx.x * MC_C;
    int ci[MC_C];
    unsigned mine = 0;  // the cases the count pass stored
#pragma unroll
    for (int k = 0; k < MC_C; ++k) {
        ci[k] = c0 + k < n ? (int)__ldg(cases + c0 + k) : 0;
        mine += c_mc_ntri[ci[k]];
    }
    unsigned total;
    const unsigned excl = mc_block_scan(mine, s_warp, total);
    unsigned long long o = tile_off[blockIdx.x] + excl;
#pragma unroll
    for (int k = 0; k < MC_C; ++k) {
        const int nt = c_mc_ntri[ci[k]];
        if (nt == 0) continue;
        const long long c = c0 + k;
        const int ii[3] = {(int)(c % cx), (int)((c / cx) % cy), (int)(c / ((long long)cx * cy))};
        float val[8];
        cube_case(phi, g, ii[0], ii[1], ii[2], val);
        mc_emit_cube(g, ii, ci[k], val, o, tris, cap);
        o += (unsigned long long)nt;
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
    const long long nt = mc_tiles(n);
    k_mc_tile_counts<<<(unsigned)nt, MC_T, 0, s>>>(phi, g, cases, tile_count);
    k_mc_tile_scan<<<1, 1024, 0, s>>>(tile_count, (int)nt, tile_off, total);
    k_mc_tile_emit<<<(unsigned)nt, MC_T, 0, s>>>(phi, g, cases, tile_off, tris, cap);
    *launches += 3;
    return cudaGetLastError();
}

}  // namespace sphk
