// sph_static.cu -- sph_bin_static: the binning of the step (cell keys,
// counting sort by cell then particle index, cell starts) for callers that
// cannot allocate device memory.
//
// Some callers are handed only their input and output buffers and must not
// call cudaMalloc: code running inside another framework's enqueue hook
// (an inference-engine plugin, a render or physics engine callback) whose
// device memory is owned by that framework's allocator and budget, or a
// real-time loop where a cudaMalloc, which may synchronise the device, would
// stall the other streams.  This entry point therefore keeps all its scratch
// (per-cell counts, per-particle ranks, scan partials, the queue of large
// cells and an error word) in one file-scope __device__ array of fixed size.
// Every GPU that loads the library holds that array until the process exits.
//
// Limits: n <= SPH_STATIC_MAX_PARTICLES and ncells <= SPH_STATIC_MAX_CELLS;
// larger requests are rejected with SPH_ERR_ARG before any device work.
// The array is shared by every call on a device and keeps the last call's
// contents; each call zeroes what must start at zero on its own stream.
// Calls that overlap on the GPU (two streams, two threads) race on the
// array: serialise them.
//
// Set-up: in host code the array's name is only a host-side stand-in, so
// every call looks up the array's device address on the current device with
// cudaGetSymbolAddress (nothing is cached: after a reset of the device's
// context the module, and the array with it, may sit at a new address).
// The first call on a device may load the module there; make that first
// call before any stream capture.
#include <math.h>
#include <stdio.h>

#include "sph_internal.cuh"

namespace {

using namespace sphk;

constexpr size_t STATIC_COUNT_OFF = 0;
constexpr size_t STATIC_PART_OFF = STATIC_COUNT_OFF + (size_t)SPH_STATIC_MAX_CELLS * 4;
constexpr size_t STATIC_PARTS = (SPH_STATIC_MAX_CELLS + 4095) / 4096 + 1;
constexpr size_t STATIC_RANK_OFF = (STATIC_PART_OFF + STATIC_PARTS * 4 + 255) & ~(size_t)255;
constexpr size_t STATIC_BIG_OFF = STATIC_RANK_OFF + (size_t)SPH_STATIC_MAX_PARTICLES * 4;
constexpr size_t STATIC_BIG_LEN = (size_t)SPH_STATIC_MAX_PARTICLES / 33 + 1;  // cells with > 32 entries
constexpr size_t STATIC_MISC_OFF = (STATIC_BIG_OFF + STATIC_BIG_LEN * 4 + 255) & ~(size_t)255;
constexpr size_t STATIC_BYTES = STATIC_MISC_OFF + 256;
static_assert(STATIC_BYTES <= SPH_STATIC_SCRATCH_BYTES, "scratch layout exceeds the declared size");

__device__ __align__(256) unsigned char g_static_scratch[SPH_STATIC_SCRATCH_BYTES];

constexpr int SORT_WARPS = 8;
constexpr int BIG_THREADS = 512;
constexpr int BIG_SMEM = 8192;  // cell entries sorted in shared memory (32 KiB)

// Compare-exchange putting the smaller value at the lower index.
__device__ __forceinline__ void cas_up(unsigned* a, int i, int j)
{
    unsigned x = a[i], y = a[j];
    if (x > y) {
        a[i] = y;
        a[j] = x;
    }
}

// Warp per cell: sort perm[start[c] .. start[c+1]) ascending in place
// (cells of up to 32 entries); larger cells are queued.
__global__ void __launch_bounds__(SORT_WARPS * 32)
k_sort_cells_index(const unsigned* __restrict__ start, int ncells, int* __restrict__ perm,
                   int* __restrict__ big_list, unsigned* __restrict__ big_count)
{
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int c = blockIdx.x * SORT_WARPS + warp;
    if (c >= ncells) return;
    unsigned s0 = start[c];
    int n = (int)(start[c + 1] - s0);
    if (n <= 1) return;
    if (n > 32) {
        if (lane == 0) big_list[atomicAdd(big_count, 1u)] = c;
        return;
    }
    int v = lane < n ? perm[s0 + lane] : 0x7fffffff;
    int r = 0;
    for (int k = 0; k < n; ++k) r += __shfl_sync(FULL, v, k) < v;
    __syncwarp();
    if (lane < n) perm[s0 + r] = v;
}

// Block per queued cell: a bitonic network whose every compare-exchange is
// ascending (the first stage of each merge compares mirrored pairs), so
// entries past n act as +infinity and need no padding.  In shared memory for
// cells up to BIG_SMEM entries, in place in global memory beyond.
__global__ void __launch_bounds__(BIG_THREADS)
k_sort_cells_index_big(const unsigned* __restrict__ start, const int* __restrict__ big_list,
                       const unsigned* __restrict__ big_count, int* __restrict__ perm)
{
    __shared__ unsigned sh[BIG_SMEM];
    const unsigned nbig = *big_count;
    for (unsigned b = blockIdx.x; b < nbig; b += gridDim.x) {
        const int c = big_list[b];
        const unsigned s0 = start[c];
        const int n = (int)(start[c + 1] - s0);
        unsigned* a = reinterpret_cast<unsigned*>(perm + s0);
        const bool in_smem = n <= BIG_SMEM;
        if (in_smem) {
            for (int e = threadIdx.x; e < n; e += BIG_THREADS) sh[e] = a[e];
            a = sh;
        }
        __syncthreads();
        int P = 1;
        while (P < n) P <<= 1;
        for (int k = 2; k <= P; k <<= 1) {
            for (int e = threadIdx.x; e < P; e += BIG_THREADS) {
                int partner = e ^ (k - 1);
                if (partner > e && partner < n) cas_up(a, e, partner);
            }
            __syncthreads();
            for (int j = k >> 2; j > 0; j >>= 1) {
                for (int e = threadIdx.x; e < P; e += BIG_THREADS) {
                    int partner = e ^ j;
                    if (partner > e && partner < n) cas_up(a, e, partner);
                }
                __syncthreads();
            }
        }
        if (in_smem) {
            unsigned* out = reinterpret_cast<unsigned*>(perm + s0);
            for (int e = threadIdx.x; e < n; e += BIG_THREADS) out[e] = sh[e];
        }
        __syncthreads();
    }
}

// Device address of the scratch array on the current device, looked up on
// every call (see the set-up note above).
int scratch_on_current_device(unsigned char** out, char* msg, size_t msg_len)
{
    void* ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
    if (e != cudaSuccess || !ptr) {
        snprintf(msg, msg_len, "cudaGetSymbolAddress of the static scratch: %s", cudaGetErrorString(e));
        return SPH_ERR_CUDA;
    }
    *out = static_cast<unsigned char*>(ptr);
    return SPH_OK;
}

thread_local char g_static_msg[512] = "";

// Failures are reported through sph_last_error(NULL), like every call made
// without a handle.
int static_fail(int code, const char* what)
{
    snprintf(g_static_msg, sizeof(g_static_msg), "%s", what);
    sphk::set_handleless_error(g_static_msg);
    return code;
}

int static_fail_msg(int code)
{
    sphk::set_handleless_error(g_static_msg);
    return code;
}

}  // namespace

extern "C" {

int sph_bin_static(const sph_params* p, int n, const float* pos4, unsigned* keys_out, int* perm_out,
                   unsigned* cell_start_out, unsigned* flags_out, void* stream)
{
    if (!p) return static_fail(SPH_ERR_ARG, "params is NULL");
    if (n < 0) return static_fail(SPH_ERR_ARG, "n < 0");
    if (n > SPH_STATIC_MAX_PARTICLES) {
        snprintf(g_static_msg, sizeof(g_static_msg),
                 "n = %d exceeds SPH_STATIC_MAX_PARTICLES = %d of the allocation-free binning", n,
                 SPH_STATIC_MAX_PARTICLES);
        return static_fail_msg(SPH_ERR_ARG);
    }
    if (!(p->cell_size > 0.0f) || !isfinite(p->cell_size)) return static_fail(SPH_ERR_ARG, "cell_size must be > 0");
    for (int a = 0; a < 3; ++a)
        if (!(isfinite(p->box_min[a]) && isfinite(p->box_max[a]) && p->box_max[a] > p->box_min[a]))
            return static_fail(SPH_ERR_ARG, "box_max must exceed box_min on every axis");
    GridDesc g;  // the grid of sph_step's binning
    const float dx = p->cell_size_x > 0.0f ? p->cell_size_x : p->cell_size;
    if (make_grid_x(p->box_min, p->box_max, dx, p->cell_size, &g) != SPH_OK || g.ncells > SPH_STATIC_MAX_CELLS) {
        snprintf(g_static_msg, sizeof(g_static_msg),
                 "the grid has more than SPH_STATIC_MAX_CELLS = %d cells", SPH_STATIC_MAX_CELLS);
        return static_fail_msg(SPH_ERR_ARG);
    }
    if (!cell_start_out || (n > 0 && (!pos4 || !keys_out || !perm_out)))
        return static_fail(SPH_ERR_ARG, "a pointer is NULL");
    if (((uintptr_t)pos4 & 15) != 0) return static_fail(SPH_ERR_ARG, "pos4 must be 16-byte aligned");
    if (((uintptr_t)flags_out & 3) != 0) return static_fail(SPH_ERR_ARG, "flags_out must be 4-byte aligned");

    unsigned char* base = nullptr;
    int rc = scratch_on_current_device(&base, g_static_msg, sizeof(g_static_msg));
    if (rc != SPH_OK) return static_fail_msg(rc);
    unsigned* count = reinterpret_cast<unsigned*>(base + STATIC_COUNT_OFF);
    unsigned* part = reinterpret_cast<unsigned*>(base + STATIC_PART_OFF);
    unsigned* rank = reinterpret_cast<unsigned*>(base + STATIC_RANK_OFF);
    int* big_list = reinterpret_cast<int*>(base + STATIC_BIG_OFF);
    unsigned* big_count = reinterpret_cast<unsigned*>(base + STATIC_MISC_OFF);
    unsigned* err = big_count + 1;

    cudaStream_t s = (cudaStream_t)stream;
    long long launches = 0;
    cudaError_t e = cudaMemsetAsync(count, 0, (size_t)g.ncells * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(big_count, 0, 8, s);
    if (e == cudaSuccess) e = launch_keys(reinterpret_cast<const float4*>(pos4), n, g, p->box_min, p->box_max,
                                          keys_out, rank, count, err, s, &launches);
    if (e == cudaSuccess) e = launch_scan(count, g.ncells, part, cell_start_out, s, &launches);
    if (e == cudaSuccess) e = launch_scatter(keys_out, rank, cell_start_out, n, perm_out, s, &launches);
    if (e == cudaSuccess) {
        k_sort_cells_index<<<(g.ncells + SORT_WARPS - 1) / SORT_WARPS, SORT_WARPS * 32, 0, s>>>(
            cell_start_out, g.ncells, perm_out, big_list, big_count);
        k_sort_cells_index_big<<<sm_count(), BIG_THREADS, 0, s>>>(cell_start_out, big_list, big_count, perm_out);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && flags_out) e = cudaMemcpyAsync(flags_out, err, 4, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) {
        snprintf(g_static_msg, sizeof(g_static_msg), "CUDA error: %s", cudaGetErrorString(e));
        return static_fail_msg(SPH_ERR_CUDA);
    }
    return SPH_OK;
}

}  // extern "C"
