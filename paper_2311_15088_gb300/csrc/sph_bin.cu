// sph_bin.cu -- uniform-grid binning of the step: cell keys with a
// warp-aggregated histogram, exclusive scan of the cell counts, scatter and
// a per-cell sort by particle id fused with the gather of the SoA state.
//
// Paper: section "Neighborhood Search" (get_cell, hash) and section
// "Neighbor Search with Sorting" (set_particle_count, prefix sum,
// count_sort_particle_index).  The paper's atomic rank makes the order
// inside a cell nondeterministic; here every cell is re-sorted by particle
// id so that the sorted order, and with it every float32 summation order,
// is a pure function of the state.
#include "sph_internal.cuh"

namespace sphk {

// ------------------------------------------------------------------ keys

struct Box {
    float box_min[3], box_max[3];
};

__global__ void __launch_bounds__(256)
k_keys(const float4* __restrict__ pos, int n, GridDesc g, Box box, unsigned* __restrict__ key,
       unsigned* __restrict__ rank, unsigned* __restrict__ count, unsigned* __restrict__ err)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    bool active = i < n;
    unsigned k = 0;
    bool clamped = false;
    if (active) {
        float4 p = pos[i];
        bool cl = false;
        k = cell_key(g, p.x, p.y, p.z, &cl);
        key[i] = k;
        clamped = outside_box(box, p.x, p.y, p.z);
    }
    unsigned r = agg_increment(count, k, active);
    if (active) rank[i] = r;
    if (__any_sync(FULL, clamped) && (threadIdx.x & 31) == 0) atomicOr(err, SPH_DEV_CLAMPED);
}

cudaError_t launch_keys(const float4* pos, int n, const GridDesc& g, const float box_min[3], const float box_max[3],
                        unsigned* key, unsigned* rank, unsigned* count, unsigned* err, cudaStream_t s,
                        long long* launches)
{
    if (n <= 0) return cudaSuccess;
    Box box;
    for (int a = 0; a < 3; ++a) {
        box.box_min[a] = box_min[a];
        box.box_max[a] = box_max[a];
    }
    k_keys<<<(n + 255) / 256, 256, 0, s>>>(pos, n, g, box, key, rank, count, err);
    ++*launches;
    return cudaGetLastError();
}

// Keys of every scene's particles: the thread of storage slot i finds its
// scene and emits the global key c_base + hash(get_cell(p)).
__global__ void __launch_bounds__(256)
k_scene_keys(const float4* __restrict__ pos, Scenes sc, unsigned* __restrict__ key,
             unsigned* __restrict__ rank, unsigned* __restrict__ count, unsigned* __restrict__ err)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    bool active = i < sc.n_all;
    unsigned k = 0;
    bool clamped = false;
    if (active) {
        const StepConst& c = sc.c[scene_of(sc.pbase, sc.S, (unsigned)i)];
        float4 p = pos[i];
        bool cl = false;
        k = (unsigned)c.c_base + cell_key(c.g, p.x, p.y, p.z, &cl);
        key[i] = k;
        // boid-attached particles follow their boids, which may leave the tank
        clamped = id_of(p) >= sc.nb_all && outside_box(c, p.x, p.y, p.z);
    }
    unsigned r = agg_increment(count, k, active);
    if (active) rank[i] = r;
    if (__any_sync(FULL, clamped) && (threadIdx.x & 31) == 0) atomicOr(err, SPH_DEV_CLAMPED);
}

cudaError_t launch_scene_keys(const float4* pos, const Scenes& sc, unsigned* key, unsigned* rank,
                              unsigned* count, unsigned* err, cudaStream_t s, long long* launches)
{
    if (sc.n_all <= 0) return cudaSuccess;
    k_scene_keys<<<(sc.n_all + 255) / 256, 256, 0, s>>>(pos, sc, key, rank, count, err);
    ++*launches;
    return cudaGetLastError();
}

// ------------------------------------------------------------------ scan

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 16;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

int scan_parts(int n) { return (n + SCAN_TILE - 1) / SCAN_TILE; }

// Block-wide exclusive scan of one value per thread; returns the block total.
__device__ __forceinline__ unsigned block_exclusive_scan(unsigned v, unsigned* prefix_out, unsigned* sh_warp)
{
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        unsigned w = lane < (SCAN_THREADS / 32) ? sh_warp[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned y = __shfl_up_sync(FULL, w, o);
            if (lane >= o) w += y;
        }
        if (lane < (SCAN_THREADS / 32)) sh_warp[lane] = w;  // inclusive warp totals
    }
    __syncthreads();
    unsigned total = sh_warp[SCAN_THREADS / 32 - 1];
    unsigned warp_base = warp ? sh_warp[warp - 1] : 0u;
    *prefix_out = warp_base + x - v;
    __syncthreads();
    return total;
}

__global__ void __launch_bounds__(SCAN_THREADS)
k_scan_reduce(const unsigned* __restrict__ in, int n, unsigned* __restrict__ part)
{
    __shared__ unsigned sh_warp[SCAN_THREADS / 32];
    int base = blockIdx.x * SCAN_TILE;
    unsigned sum = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        int idx = base + k * SCAN_THREADS + threadIdx.x;
        if (idx < n) sum += in[idx];
    }
    unsigned dummy;
    unsigned total = block_exclusive_scan(sum, &dummy, sh_warp);
    if (threadIdx.x == 0) part[blockIdx.x] = total;
}

// One block: exclusive scan of the tile totals in place; part[nparts] =
// total.  1024 values per round: a shuffle scan in each warp, then of the
// 32 warp totals by the first warp.
__global__ void __launch_bounds__(1024) k_scan_parts(unsigned* __restrict__ part, int nparts)
{
    __shared__ unsigned sh_w[32];
    __shared__ unsigned carry_sh;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned carry = 0;
    for (int base = 0; base < nparts; base += 1024) {
        const int idx = base + threadIdx.x;
        const unsigned v = idx < nparts ? part[idx] : 0u;
        unsigned x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(FULL, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) sh_w[warp] = x;
        __syncthreads();
        if (warp == 0) {
            unsigned w = sh_w[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned y = __shfl_up_sync(FULL, w, o);
                if (lane >= o) w += y;
            }
            sh_w[lane] = w;  // inclusive warp totals
            if (lane == 31) carry_sh = w;
        }
        __syncthreads();
        const unsigned incl = x + (warp ? sh_w[warp - 1] : 0u);
        if (idx < nparts) part[idx] = carry + incl - v;
        carry += carry_sh;
        __syncthreads();
    }
    if (threadIdx.x == 0) part[nparts] = carry;
}

// Element e of a tile lives at sh[e + e / 32]: one padding word per 32
// keeps both the coalesced phase (thread t, elements k * 256 + t) and the
// per-thread phase (thread t, elements 16 t .. 16 t + 15) free of bank
// conflicts (without it the second phase is a 16-way conflict).
__device__ __forceinline__ int scan_pad(int e) { return e + (e >> 5); }

__global__ void __launch_bounds__(SCAN_THREADS)
k_scan_tiles(const unsigned* __restrict__ in, int n, const unsigned* __restrict__ part,
             unsigned* __restrict__ out)
{
    __shared__ unsigned sh[SCAN_TILE + SCAN_TILE / 32];
    __shared__ unsigned sh_warp[SCAN_THREADS / 32];
    int base = blockIdx.x * SCAN_TILE;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        int idx = base + k * SCAN_THREADS + threadIdx.x;
        sh[scan_pad(k * SCAN_THREADS + threadIdx.x)] = idx < n ? in[idx] : 0u;
    }
    __syncthreads();
    unsigned local[SCAN_ITEMS];
    unsigned sum = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        local[k] = sh[scan_pad(threadIdx.x * SCAN_ITEMS + k)];
        sum += local[k];
    }
    unsigned prefix;
    block_exclusive_scan(sum, &prefix, sh_warp);
    prefix += part[blockIdx.x];
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        sh[scan_pad(threadIdx.x * SCAN_ITEMS + k)] = prefix;
        prefix += local[k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        int idx = base + k * SCAN_THREADS + threadIdx.x;
        if (idx < n) out[idx] = sh[scan_pad(k * SCAN_THREADS + threadIdx.x)];
    }
}

__global__ void k_scan_total(const unsigned* __restrict__ part, int nparts, unsigned* __restrict__ out, int n)
{
    out[n] = part[nparts];
}

cudaError_t launch_scan(const unsigned* counts, int n, unsigned* part, unsigned* start,
                        cudaStream_t s, long long* launches)
{
    if (n <= 0) return cudaSuccess;
    int np = scan_parts(n);
    k_scan_reduce<<<np, SCAN_THREADS, 0, s>>>(counts, n, part);
    k_scan_parts<<<1, 1024, 0, s>>>(part, np);
    k_scan_tiles<<<np, SCAN_THREADS, 0, s>>>(counts, n, part, start);
    k_scan_total<<<1, 1, 0, s>>>(part, np, start, n);
    *launches += 4;
    return cudaGetLastError();
}

// --------------------------------------------------------------- scatter

__global__ void __launch_bounds__(256)
k_scatter(const unsigned* __restrict__ key, const unsigned* __restrict__ rank,
          const unsigned* __restrict__ start, int n, int* __restrict__ tmp)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) tmp[start[key[i]] + rank[i]] = i;
}

// The same, also placing each particle's id (pos.w) beside its index:
// tmp_id[start[key] + rank] = id, so that the per-cell sort ranks a cell's
// particles from one contiguous run of ids.
__global__ void __launch_bounds__(256)
k_scatter_ids(const unsigned* __restrict__ key, const unsigned* __restrict__ rank,
              const unsigned* __restrict__ start, const float4* __restrict__ pos, int n, int* __restrict__ tmp,
              int* __restrict__ tmp_id)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const unsigned dst = start[key[i]] + rank[i];
    tmp[dst] = i;
    tmp_id[dst] = id_of(pos[i]);
}

cudaError_t launch_scatter_ids(const unsigned* key, const unsigned* rank, const unsigned* start, const float4* pos,
                               int n, int* tmp, int* tmp_id, cudaStream_t s, long long* launches)
{
    if (n <= 0) return cudaSuccess;
    k_scatter_ids<<<(n + 255) / 256, 256, 0, s>>>(key, rank, start, pos, n, tmp, tmp_id);
    ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_scatter(const unsigned* key, const unsigned* rank, const unsigned* start, int n,
                           int* tmp, cudaStream_t s, long long* launches)
{
    if (n <= 0) return cudaSuccess;
    k_scatter<<<(n + 255) / 256, 256, 0, s>>>(key, rank, start, n, tmp);
    ++*launches;
    return cudaGetLastError();
}

// ------------------------------------------------ per-cell sort + gather

constexpr int SORT_WARPS = 8;
constexpr int SORT_SMEM = 128;     // cells up to this size are ranked by one warp
constexpr int BIG_THREADS = 1024;  // larger cells: one block, bitonic sort in smem
constexpr int BIG_CAP = 16384;     // elements of a block sort (128 KiB of smem)
// blocks of k_cellsort_big: one per multiprocessor (they loop over the queued cells)

// One warp per cell.  tmp[start[c] ..) holds the storage indices of the
// cell's particles in arbitrary order; each is ranked by particle id and its
// pos/vel copied to start[c] + rank.  The attached particle of boid b
// records its sorted slot in slot_of_boid[b].  Cells with more than
// SORT_SMEM entries are queued in big_list for k_cellsort_big.
__global__ void __launch_bounds__(SORT_WARPS * 32)
k_cellsort_gather(const unsigned* __restrict__ start, int ncells, const int* __restrict__ tmp,
                  const float4* __restrict__ pos_in, const float4* __restrict__ vel_in,
                  float4* __restrict__ pos_out, float4* __restrict__ vel_out, int nb,
                  int* __restrict__ slot_of_boid, int* __restrict__ big_list, unsigned* __restrict__ big_count)
{
    __shared__ int sh_id[SORT_WARPS][SORT_SMEM];
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int c = blockIdx.x * SORT_WARPS + warp;
    if (c >= ncells) return;
    unsigned s0 = start[c];
    int n = (int)(start[c + 1] - s0);
    if (n == 0) return;
    if (n <= 32) {
        int src = 0, id = 0x7fffffff;
        if (lane < n) {
            src = tmp[s0 + lane];
            id = id_of(pos_in[src]);
        }
        int r = 0;
        for (int k = 0; k < n; ++k) {
            int o = __shfl_sync(FULL, id, k);
            r += o < id;
        }
        if (lane < n) {
            unsigned dst = s0 + (unsigned)r;
            pos_out[dst] = pos_in[src];
            vel_out[dst] = vel_in[src];
            if (id < nb && slot_of_boid) slot_of_boid[id] = (int)dst;
        }
        return;
    }
    if (n > SORT_SMEM) {
        if (lane == 0) big_list[atomicAdd(big_count, 1u)] = c;
        return;
    }
    for (int e = lane; e < n; e += 32) sh_id[warp][e] = id_of(pos_in[tmp[s0 + e]]);
    __syncwarp();
    for (int e = lane; e < n; e += 32) {
        int src = tmp[s0 + e];
        int id = sh_id[warp][e];
        int r = 0;
        for (int k = 0; k < n; ++k) r += sh_id[warp][k] < id;
        unsigned dst = s0 + (unsigned)r;
        pos_out[dst] = pos_in[src];
        vel_out[dst] = vel_in[src];
        if (id < nb && slot_of_boid) slot_of_boid[id] = (int)dst;
    }
}

// One block per queued large cell: (id, storage index) pairs sorted by a
// bitonic network in shared memory, then gathered.  Cells beyond BIG_CAP are
// ranked by counting straight from global memory.
__global__ void __launch_bounds__(BIG_THREADS)
k_cellsort_big(const unsigned* __restrict__ start, const int* __restrict__ big_list,
               const unsigned* __restrict__ big_count, const int* __restrict__ tmp,
               const float4* __restrict__ pos_in, const float4* __restrict__ vel_in,
               float4* __restrict__ pos_out, float4* __restrict__ vel_out, int nb,
               int* __restrict__ slot_of_boid, const int* __restrict__ tmp_id, float* __restrict__ soa,
               size_t soa_st)
{
    extern __shared__ unsigned long long sh_kv[];
    // id of the entry at sorted-scratch position e (from tmp_id when given)
    auto id_at = [&](unsigned e) { return tmp_id ? tmp_id[e] : id_of(pos_in[tmp[e]]); };
    auto put = [&](unsigned dst, int src) {
        const float4 p = pos_in[src];
        pos_out[dst] = p;
        vel_out[dst] = vel_in[src];
        if (soa) {
            soa[dst] = p.x;
            soa[soa_st + dst] = p.y;
            soa[2 * soa_st + dst] = p.z;
        }
    };
    const unsigned nbig = *big_count;
    for (unsigned b = blockIdx.x; b < nbig; b += gridDim.x) {
        const int c = big_list[b];
        const unsigned s0 = start[c];
        const int n = (int)(start[c + 1] - s0);
        if (n <= BIG_CAP) {
            int P = 1;
            while (P < n) P <<= 1;
            for (int e = threadIdx.x; e < P; e += BIG_THREADS) {
                unsigned long long v = ~0ull;
                if (e < n) {
                    int src = tmp[s0 + e];
                    v = ((unsigned long long)(unsigned)id_at(s0 + e) << 32) | (unsigned)src;
                }
                sh_kv[e] = v;
            }
            __syncthreads();
            for (int k = 2; k <= P; k <<= 1) {
                for (int j = k >> 1; j > 0; j >>= 1) {
                    for (int e = threadIdx.x; e < P; e += BIG_THREADS) {
                        int partner = e ^ j;
                        if (partner > e) {
                            unsigned long long x = sh_kv[e], y = sh_kv[partner];
                            bool ascending = (e & k) == 0;
                            if ((x > y) == ascending) {
                                sh_kv[e] = y;
                                sh_kv[partner] = x;
                            }
                        }
                    }
                    __syncthreads();
                }
            }
            for (int e = threadIdx.x; e < n; e += BIG_THREADS) {
                unsigned long long v = sh_kv[e];
                int src = (int)(unsigned)(v & 0xffffffffull);
                int id = (int)(unsigned)(v >> 32);
                unsigned dst = s0 + (unsigned)e;
                put(dst, src);
                if (id < nb && slot_of_boid) slot_of_boid[id] = (int)dst;
            }
        } else {
            for (int e = threadIdx.x; e < n; e += BIG_THREADS) {
                int src = tmp[s0 + e];
                int id = id_at(s0 + e);
                int r = 0;
                for (int k = 0; k < n; ++k) r += id_at(s0 + k) < id;
                unsigned dst = s0 + (unsigned)r;
                put(dst, src);
                if (id < nb && slot_of_boid) slot_of_boid[id] = (int)dst;
            }
        }
        __syncthreads();
    }
}

// One-time kernel attributes (the block sort's 128 KiB of shared memory);
// called when a handle is created, before any stream capture.
cudaError_t prepare_kernels()
{
    static bool done = false;
    if (done) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_cellsort_big, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         BIG_CAP * (int)sizeof(unsigned long long));
    if (e == cudaSuccess) done = true;
    return e;
}

cudaError_t launch_cellsort_gather(const unsigned* start, int ncells, const int* tmp,
                                   const float4* pos_in, const float4* vel_in, float4* pos_out,
                                   float4* vel_out, int nb, int* slot_of_boid, int* big_list,
                                   unsigned* big_count, cudaStream_t s, long long* launches)
{
    if (ncells <= 0) return cudaSuccess;
    cudaError_t e = prepare_kernels();
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(big_count, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    int blocks = (ncells + SORT_WARPS - 1) / SORT_WARPS;
    k_cellsort_gather<<<blocks, SORT_WARPS * 32, 0, s>>>(start, ncells, tmp, pos_in, vel_in, pos_out,
                                                         vel_out, nb, slot_of_boid, big_list, big_count);
    k_cellsort_big<<<sm_count(), BIG_THREADS, BIG_CAP * sizeof(unsigned long long), s>>>(
        start, big_list, big_count, tmp, pos_in, vel_in, pos_out, vel_out, nb, slot_of_boid, nullptr, nullptr, 0);
    *launches += 2;
    return cudaGetLastError();
}

// One thread per sorted slot: the thread of slot s takes the storage index
// tmp[s] of its cell, ranks its id tmp_id[s] against the cell's other ids
// (a contiguous run of tmp_id) and moves pos/vel to start[c] + rank, also
// writing x, y, z to the SoA copy (soa, soa_st floats per axis).  Cells with
// more than SLOT_SMALL entries are queued (by the thread of their first
// slot) for k_cellsort_big.  Suited to grids of small cells (a few particles
// each).
constexpr int SLOT_SMALL = 128;  // compressed fluid fills h/2 cells with 60-100 particles

__global__ void __launch_bounds__(256)
k_cellsort_slots(const unsigned* __restrict__ start, const unsigned* __restrict__ key, int n,
                 const int* __restrict__ tmp, const int* __restrict__ tmp_id, const float4* __restrict__ pos_in,
                 const float4* __restrict__ vel_in, float4* __restrict__ pos_out,
                 float4* __restrict__ vel_out, float* __restrict__ soa, size_t soa_st, int nb,
                 int* __restrict__ slot_of_boid, int* __restrict__ big_list, unsigned* __restrict__ big_count)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int src = tmp[s];
    const unsigned c = key[src];
    const unsigned s0 = start[c];
    const int nc = (int)(start[c + 1] - s0);
    if (nc > SLOT_SMALL) {
        if ((unsigned)s == s0) big_list[atomicAdd(big_count, 1u)] = (int)c;
        return;
    }
    const int id = tmp_id[s];
    int r = 0;
    for (int k = 0; k < nc; ++k) r += __ldg(tmp_id + s0 + k) < id;
    const unsigned dst = s0 + (unsigned)r;
    const float4 p = pos_in[src];
    pos_out[dst] = p;
    vel_out[dst] = vel_in[src];
    soa[dst] = p.x;
    soa[soa_st + dst] = p.y;
    soa[2 * soa_st + dst] = p.z;
    if (id < nb && slot_of_boid) slot_of_boid[id] = (int)dst;
}

cudaError_t launch_cellsort_slots(const unsigned* start, const unsigned* key, int n, int ncells,
                                  const int* tmp, const int* tmp_id, const float4* pos_in, const float4* vel_in,
                                  float4* pos_out, float4* vel_out, float* soa, int nb, int* slot_of_boid,
                                  int* big_list, unsigned* big_count, cudaStream_t s, long long* launches)
{
    if (n <= 0 || ncells <= 0) return cudaSuccess;
    cudaError_t e = prepare_kernels();
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(big_count, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    const size_t st = soa_stride((size_t)n);
    k_cellsort_slots<<<(n + 255) / 256, 256, 0, s>>>(start, key, n, tmp, tmp_id, pos_in, vel_in, pos_out, vel_out,
                                                     soa, st, nb, slot_of_boid, big_list, big_count);
    k_cellsort_big<<<sm_count(), BIG_THREADS, BIG_CAP * sizeof(unsigned long long), s>>>(
        start, big_list, big_count, tmp, pos_in, vel_in, pos_out, vel_out, nb, slot_of_boid, tmp_id, soa, st);
    *launches += 2;
    return cudaGetLastError();
}

// Key of every sorted slot, recovered from cell_start (warp per cell).
__global__ void __launch_bounds__(256)
k_slot_keys(const unsigned* __restrict__ start, int ncells, unsigned* __restrict__ slot_key)
{
    int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (c >= ncells) return;
    for (unsigned s = start[c] + lane; s < start[c + 1]; s += 32) slot_key[s] = (unsigned)c;
}

cudaError_t launch_slot_keys(const unsigned* start, int ncells, unsigned* slot_key, cudaStream_t s,
                             long long* launches)
{
    if (ncells <= 0) return cudaSuccess;
    k_slot_keys<<<(ncells + 7) / 8, 256, 0, s>>>(start, ncells, slot_key);
    ++*launches;
    return cudaGetLastError();
}

}  // namespace sphk
