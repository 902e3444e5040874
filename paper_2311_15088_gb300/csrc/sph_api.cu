// sph_api.cu -- the C ABI declared in include/sph.h: parameter validation,
// the workspace layout, state upload/download, step orchestration and the
// field accessors.  All device work is enqueued on the caller's stream;
// nothing here allocates device memory.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <new>

#include "sph_internal.cuh"

using namespace sphk;

struct sph_handle {
    int S;                    // scenes (1 for sph_create)
    sph_params* params;       // host copies, S entries
    StepConst* consts;        // host copies, S entries
    unsigned *h_pbase, *h_bbase;
    StepConst* d_consts;      // device copies (in the workspace)
    unsigned *d_pbase, *d_bbase;
    Scenes sc;                // what the kernels receive
    Tuning tune;
    int n_fluid, n_boid, n;   // totals over the scenes
    int ncells, nbcells;      // totals over the scenes
    int nfcells;              // cells of the surrogate's feature grids
    int4* fgrid;              // their integer sums (count, velocity in 2^-16 fixed point)
    // state (storage order) and the sorted scratch copy
    float4 *pos, *vel, *pos_s, *vel_s;
    float* soa;               // pos_s as three float arrays (x, y, z), soa_stride(n) each
    unsigned *key, *rank;
    int* tmp;
    int* tmp_id;              // ids beside tmp (the per-cell sort's ranking keys)
    unsigned *count, *cell_start, *scan_part;
    int* big_list;
    unsigned* big_count;
    float* rho;
    float2* ab;  // (m / rho, p) per sorted slot
    int* nbr;
    float4* prec;             // the force pass's pair record of each sorted slot (2 float4)
    uint2* seg;               // hit segments of the density pass (SEG_CAP per particle)
    unsigned* pipe_queue;     // the fused pipeline's work counters and barrier (3 words)
    int skip_cta;             // test hook of the pipeline's barrier (-1: off)
    int* nseg;
    int* ncand;
    float4* acc;
    int* touched;
    float4* infl;
    int* slot_of_boid;
    float4 *bpos, *bvel, *bpos_s, *bvel_s;
    unsigned *bkey, *brank;
    int* btmp;
    unsigned *bcount, *bstart, *bscan_part;
    int* bbig_list;
    unsigned* bbig_count;
    float4* fb;
    float4* obst;             // obstacle grid over the boid grid (nbcells)
    float* obst_shapes;       // spheres then boxes (SPH_MAX_OBSTACLES x 10 floats)
    unsigned* err;
    // surrogate: features, network output, exact-path masks
    void* feat;               // BF16 [nb_pad][SPH_MLP_IN]
    float* yout;              // [nb_pad][SPH_MLP_OUT]
    unsigned char* need;
    int* need_list;     // compacted slots whose density a boid force needs
    unsigned* need_len;
    unsigned* noff;        // neighbour-list offsets (n + 1) and scan partials
    unsigned* noff_part;
    unsigned* list;        // the caller's pair buffer (NULL: no lists)
    size_t list_cap;      // per sorted slot
    int* bflag;               // per boid
    int nb_pad;
    int stats_chunks;         // blocks per scene of the statistics (sph_stats)
    double* stats_part;       // their float64 partials
    double* stats_out;        // staging of a host copy (S x SPH_STATS_N)
    sph_mlp* mlp;
    float f_scale, log_err_max;
    const float *feat_lo, *feat_hi;  // the caller's input range (NULL: no check)
    bool has_state, keys_ready, has_step;
    bool diag;                // record acc, touched, influence in the step (sph_set_diagnostics)
    bool diag_step;           // the most recent step recorded them
    long long launches;
    cudaStream_t last_stream;
    // per-pass event timing (sph_profile_enable)
    cudaEvent_t* prof_ev;
    int* prof_kind;
    int prof_cap, prof_n;
    // the step's side stream: the boids' binning, F_b and rules run there,
    // alongside the fluid passes (forked from and joined back into the
    // caller's stream every step)
    cudaStream_t side;
    cudaEvent_t ev_fork, ev_dens, ev_join;
    // captured step (sph_graph_step)
    cudaGraphExec_t graph;
    cudaStream_t graph_stream;
    long long graph_launches;
    // captured boid-force calls (sph_graph_boid_forces), one per mode
    struct {
        cudaGraphExec_t exec;
        cudaStream_t stream;
        float* out;
        long long launches;
        bool warm;  // one plain call of this mode has run (one-time set-up done)
    } bgraph[4];
    char msg[512];
};

static void drop_boid_graphs(sph_handle* h)
{
    for (auto& g : h->bgraph) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        g.exec = nullptr;
    }
}

static void destroy_side(sph_handle* h)
{
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_dens) cudaEventDestroy(h->ev_dens);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    if (h->side) cudaStreamDestroy(h->side);
    h->ev_fork = h->ev_dens = h->ev_join = nullptr;
    h->side = nullptr;
}

static void prof_begin(sph_handle* h, int kind, cudaStream_t s)
{
    if (h->prof_n < h->prof_cap) {
        cudaEventRecord(h->prof_ev[2 * h->prof_n], s);
        h->prof_kind[h->prof_n] = kind;
    }
}

static void prof_end(sph_handle* h, cudaStream_t s)
{
    if (h->prof_n < h->prof_cap) {
        cudaEventRecord(h->prof_ev[2 * h->prof_n + 1], s);
        ++h->prof_n;
    }
}

static thread_local char g_msg[512] = "";

int sphk::sm_count()
{
    static std::atomic<int> cache[64];  // per device ordinal; 0 = not queried yet
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return 1;
    if (dev >= 64) {
        int v = 0;
        return cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0 ? v : 1;
    }
    int v = cache[dev].load(std::memory_order_relaxed);
    if (v <= 0) {
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) return 1;
        cache[dev].store(v, std::memory_order_relaxed);
    }
    return v;
}

void sphk::set_handleless_error(const char* msg) { snprintf(g_msg, sizeof(g_msg), "%s", msg); }

static int fail(sph_handle* h, int code, const char* fmt, ...)
{
    char* dst = h ? h->msg : g_msg;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(dst, 512, fmt, ap);
    va_end(ap);
    return code;
}

#define CUDA_TRY(h, expr)                                                                   \
    do {                                                                                    \
        cudaError_t e_ = (expr);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return fail((h), SPH_ERR_CUDA, "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_),  \
                        __FILE__, __LINE__);                                                \
    } while (0)

// ------------------------------------------------------------ parameters

static bool finite_pos(float v) { return isfinite(v) && v > 0.0f; }

int sphk::make_grid_x(const float mn[3], const float mx[3], float dx, float d, GridDesc* g)
{
    long long cells = 1;
    for (int a = 0; a < 3; ++a) {
        double n = ceil(((double)mx[a] - (double)mn[a]) / (double)(a == 0 ? dx : d));
        if (n < 1.0) n = 1.0;
        if (n > 2147483647.0) return SPH_ERR_OVERFLOW;
        g->dim[a] = (int)n;
        g->minf[a] = mn[a];
        cells *= (long long)n;
        if (cells > 2147483646LL) return SPH_ERR_OVERFLOW;
    }
    g->ncells = (int)cells;
    g->inv_d = 1.0f / d;
    g->inv_dx = 1.0f / dx;
    return SPH_OK;
}

// The particle grid's cell size along x (cell_size_x, 0: cell_size).
static float cell_x(const sph_params* p) { return p->cell_size_x > 0.0f ? p->cell_size_x : p->cell_size; }

static int validate(const sph_params* p, int n_fluid, int n_boid)
{
    if (!p) return fail(nullptr, SPH_ERR_ARG, "params is NULL");
    if (n_fluid < 0 || n_boid < 0) return fail(nullptr, SPH_ERR_ARG, "negative particle count");
    if ((long long)n_fluid + n_boid > 2147483647LL) return fail(nullptr, SPH_ERR_OVERFLOW, "too many particles");
    if (!finite_pos(p->h) || !finite_pos(p->rho0) || !finite_pos(p->mass) || !finite_pos(p->dt))
        return fail(nullptr, SPH_ERR_ARG, "h, rho0, mass and dt must be finite and > 0");
    if (!(isfinite(p->cell_size) && p->cell_size >= 0.25f * p->h))
        return fail(nullptr, SPH_ERR_ARG, "cell_size must be >= h/4");
    if (!(isfinite(p->cell_size_x) && (p->cell_size_x == 0.0f || p->cell_size_x >= 0.125f * p->h)))
        return fail(nullptr, SPH_ERR_ARG, "cell_size_x must be 0 or >= h/8");
    if (!(isfinite(p->k) && p->k >= 0.0f) || !(isfinite(p->mu) && p->mu >= 0.0f))
        return fail(nullptr, SPH_ERR_ARG, "k and mu must be finite and >= 0");
    for (int a = 0; a < 3; ++a)
        if (!(isfinite(p->box_min[a]) && isfinite(p->box_max[a]) && p->box_max[a] > p->box_min[a]))
            return fail(nullptr, SPH_ERR_ARG, "box_max must exceed box_min on every axis");
    if (!(isfinite(p->gx) && isfinite(p->gy) && isfinite(p->gz)))
        return fail(nullptr, SPH_ERR_ARG, "gravity must be finite");
    if (p->const_set != SPH_MULLER3D && p->const_set != SPH_PAPER_LITERAL)
        return fail(nullptr, SPH_ERR_ARG, "unknown const_set %d", p->const_set);
    if (p->coupling_mode != SPH_COUPLE_FORCE && p->coupling_mode != SPH_COUPLE_LITERAL)
        return fail(nullptr, SPH_ERR_ARG, "unsupported coupling_mode %d", p->coupling_mode);
    if (!(isfinite(p->wall_restitution) && p->wall_restitution >= 0.0f))
        return fail(nullptr, SPH_ERR_ARG, "wall_restitution must be >= 0");
    if (!(p->r_sep >= 0.0f && p->r_vis >= p->r_sep && isfinite(p->r_vis)))
        return fail(nullptr, SPH_ERR_ARG, "need 0 <= r_sep <= r_vis");
    if (!(isfinite(p->boid_cell_size) && p->boid_cell_size > 0.0f && p->boid_cell_size >= 0.25f * p->r_vis))
        return fail(nullptr, SPH_ERR_ARG, "boid_cell_size must be > 0 and >= r_vis/4");
    if (!(p->v_min >= 0.0f && p->v_max >= p->v_min && isfinite(p->v_max)))
        return fail(nullptr, SPH_ERR_ARG, "need 0 <= v_min <= v_max");
    if (!(isfinite(p->w_sep) && isfinite(p->w_align) && isfinite(p->w_coh) && isfinite(p->sph_factor) &&
          isfinite(p->edge_turn)))
        return fail(nullptr, SPH_ERR_ARG, "boid weights must be finite");
    GridDesc g;
    if (make_grid_x(p->box_min, p->box_max, cell_x(p), p->cell_size, &g) != SPH_OK)
        return fail(nullptr, SPH_ERR_OVERFLOW, "particle grid has more than 2^31 cells");
    if (make_grid(p->box_min, p->box_max, p->boid_cell_size, &g) != SPH_OK)
        return fail(nullptr, SPH_ERR_OVERFLOW, "boid grid has more than 2^31 cells");
    return SPH_OK;
}

// Search bounds of a walk with radius^2 r2 (the float32 predicate bound) on
// cells of size d: reach2 = r2 (1 + 1e-5) exceeds the exact squared
// distance of any pair that passes the float32 predicate, and margin covers
// the rounding of cell boundaries (8 ulps of the largest coordinate + 1e-5 d).
static WalkBounds make_bounds(const sph_params* p, float r2, float d, float dx)
{
    float extent = d;
    for (int a = 0; a < 3; ++a) extent = fmaxf(extent, fmaxf(fabsf(p->box_min[a]), fabsf(p->box_max[a])) + d);
    const float ulp = nextafterf(extent, INFINITY) - extent;
    WalkBounds w;
    w.margin = 8.0f * ulp + 1e-5f * fminf(d, dx);
    w.reach2 = r2 * (1.0f + 1e-5f);
    w.reach = sqrtf(w.reach2) + w.margin;
    w.d = d;
    return w;
}

static void make_const(const sph_params* p, int n_fluid, int n_boid, StepConst* c)
{
    memset(c, 0, sizeof(*c));
    make_grid_x(p->box_min, p->box_max, cell_x(p), p->cell_size, &c->g);
    make_grid(p->box_min, p->box_max, p->boid_cell_size, &c->gb);
    c->wg = make_bounds(p, p->h * p->h, p->cell_size, cell_x(p));
    c->wb = make_bounds(p, p->r_vis * p->r_vis, p->boid_cell_size, p->boid_cell_size);
    c->n = n_fluid + n_boid;
    c->nb = n_boid;  // bases and nb_all are filled in by layout_scenes
    const double pi = 3.14159265358979323846;
    const double h = p->h;
    c->h2 = p->h * p->h;
    c->mC6 = (float)((double)p->mass * 315.0 / (64.0 * pi * pow(h, 9)));
    double cp, cv;
    if (p->const_set == SPH_PAPER_LITERAL) {
        cp = 30.0 / (pi * pow(h, 4));
        cv = 40.0 / (pi * pow(h, 4));
    } else {
        cp = 45.0 / (pi * pow(h, 5));
        cv = cp;
    }
    c->half_cp_h = (float)(0.5 * cp * h);
    c->cv_mu = (float)(cv * (double)p->mu);
    c->h = p->h;
    c->inv_h = (float)(1.0 / h);
    c->mass = p->mass;
    c->k = p->k;
    c->rho0 = p->rho0;
    c->dt = p->dt;
    c->grav[0] = p->gx;
    c->grav[1] = p->gy;
    c->grav[2] = p->gz;
    for (int a = 0; a < 3; ++a) {
        c->box_min[a] = p->box_min[a];
        c->box_max[a] = p->box_max[a];
    }
    c->restitution = p->wall_restitution;
    c->rs = p->r_sep;
    c->rs2 = p->r_sep * p->r_sep;
    c->rv2 = p->r_vis * p->r_vis;
    c->w_sep = p->w_sep;
    c->w_align = p->w_align;
    c->w_coh = p->w_coh;
    c->sph_dt = (float)((double)p->sph_factor * (double)p->dt);
    c->sph_factor = p->sph_factor;
    c->literal = p->coupling_mode == SPH_COUPLE_LITERAL;
    for (int a = 0; a < 3; ++a)  // the highest feature cell of a position in the box, plus margins
        c->fdim[a] = (int)floorf((p->box_max[a] - p->box_min[a]) * c->inv_h) + 1 + 4;
    c->v_min = p->v_min;
    c->v_max = p->v_max;
    c->edge_turn = p->edge_turn;
}

// ------------------------------------------------------------- workspace

struct Carver {
    uintptr_t base, off;
    template <class T>
    T* take(size_t count)
    {
        off = (off + 255) & ~(uintptr_t)255;
        T* ptr = reinterpret_cast<T*>(base + off);
        off += count * sizeof(T) + 16;  // + guard so that empty arrays stay distinct
        return ptr;
    }
};

static size_t carve(sph_handle* h, uintptr_t base)
{
    Carver cv{base, 0};
    const size_t n = (size_t)h->n, nb = (size_t)h->n_boid;
    const size_t C = (size_t)h->ncells, Cb = (size_t)h->nbcells;
    h->d_consts = cv.take<StepConst>((size_t)h->S);
    h->d_pbase = cv.take<unsigned>((size_t)h->S + 1);
    h->d_bbase = cv.take<unsigned>((size_t)h->S + 1);
    h->pos = cv.take<float4>(n);
    h->vel = cv.take<float4>(n);
    h->pos_s = cv.take<float4>(n);
    h->vel_s = cv.take<float4>(n);
    h->soa = cv.take<float>(3 * soa_stride(n));
    h->key = cv.take<unsigned>(n);
    h->rank = cv.take<unsigned>(n);
    h->tmp = cv.take<int>(n > C ? n : C);
    h->tmp_id = cv.take<int>(n);
    h->count = cv.take<unsigned>(C);
    h->cell_start = cv.take<unsigned>(C + 1);
    h->scan_part = cv.take<unsigned>((size_t)scan_parts((int)C) + 1);
    h->big_list = cv.take<int>(C);
    h->big_count = cv.take<unsigned>(1);
    h->rho = cv.take<float>(n);
    h->ab = cv.take<float2>(n);
    h->nbr = cv.take<int>(n);
    h->prec = cv.take<float4>(2 * n);
    h->pipe_queue = cv.take<unsigned>(4);
    h->fgrid = cv.take<int4>((size_t)h->nfcells);
    h->seg = cv.take<uint2>(n * (size_t)SEG_CAP);
    h->nseg = cv.take<int>(n);
    h->ncand = cv.take<int>(n);
    h->acc = cv.take<float4>(n);
    h->touched = cv.take<int>(n);
    h->infl = cv.take<float4>(n);
    h->slot_of_boid = cv.take<int>(nb);
    h->bpos = cv.take<float4>(nb);
    h->bvel = cv.take<float4>(nb);
    h->bpos_s = cv.take<float4>(nb);
    h->bvel_s = cv.take<float4>(nb);
    h->bkey = cv.take<unsigned>(nb);
    h->brank = cv.take<unsigned>(nb);
    h->btmp = cv.take<int>(nb > Cb ? nb : Cb);
    h->bcount = cv.take<unsigned>(Cb);
    h->bstart = cv.take<unsigned>(Cb + 1);
    h->bscan_part = cv.take<unsigned>((size_t)scan_parts((int)Cb) + 1);
    h->bbig_list = cv.take<int>(Cb);
    h->bbig_count = cv.take<unsigned>(1);
    h->fb = cv.take<float4>(nb);
    h->obst = cv.take<float4>(Cb);
    h->obst_shapes = cv.take<float>((size_t)SPH_MAX_OBSTACLES * 10);
    h->err = cv.take<unsigned>(4);
    h->nb_pad = nb ? (int)((nb + 127) / 128 * 128) : 0;
    h->feat = cv.take<unsigned short>((size_t)h->nb_pad * SPH_MLP_IN);
    h->yout = cv.take<float>((size_t)h->nb_pad * SPH_MLP_OUT);
    h->need = cv.take<unsigned char>(n);
    h->need_list = cv.take<int>(n);
    h->need_len = cv.take<unsigned>(1);
    h->noff = cv.take<unsigned>(n + 1);
    h->noff_part = cv.take<unsigned>((size_t)scan_parts((int)n) + 1);
    h->bflag = cv.take<int>(nb);
    h->stats_part = cv.take<double>((size_t)h->S * h->stats_chunks * STATS_PART);
    h->stats_out = cv.take<double>((size_t)h->S * STATS_OUT);
    return (size_t)((cv.off + 255) & ~(uintptr_t)255);
}

// ---------------------------------------------------------- state kernels

// Storage slot i of scene k: its first n_boid(k) slots hold the scene's
// attached particles, then its fluid particles.  Attached particle of global
// boid b gets id b; fluid particle f (global fluid index) gets id nb_all + f.
__global__ void k_load_state(const float4* __restrict__ fpos, const float4* __restrict__ fvel,
                             const float4* __restrict__ bpos_in, const float4* __restrict__ bvel_in,
                             Scenes sc, float4* __restrict__ pos, float4* __restrict__ vel,
                             float4* __restrict__ bpos, float4* __restrict__ bvel, int* __restrict__ slot_of_boid)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= sc.n_all) return;
    const int k = scene_of(sc.pbase, sc.S, (unsigned)i);
    const unsigned local = (unsigned)i - sc.pbase[k];
    const unsigned nbk = sc.bbase[k + 1] - sc.bbase[k];
    float4 p, v;
    if (local < nbk) {
        const int b = (int)(sc.bbase[k] + local);
        p = bpos_in[b];
        v = bvel_in[b];
        p.w = __int_as_float(b);
        v.w = 0.0f;
        bpos[b] = p;
        bvel[b] = v;
        slot_of_boid[b] = i;
    } else {
        const int f = (int)(sc.pbase[k] - sc.bbase[k] + (local - nbk));
        p = fpos[f];
        v = fvel[f];
        p.w = __int_as_float(sc.nb_all + f);
        v.w = 0.0f;
    }
    pos[i] = p;
    vel[i] = v;
}

__global__ void k_store_state(const float4* __restrict__ pos, const float4* __restrict__ vel,
                              const float4* __restrict__ bpos, const float4* __restrict__ bvel, int n, int nb,
                              float4* __restrict__ fpos, float4* __restrict__ fvel, float4* __restrict__ opos,
                              float4* __restrict__ ovel)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        float4 p = pos[i];
        int id = __float_as_int(p.w);
        if (id >= nb) {
            float4 v = vel[i];
            fpos[id - nb] = make_float4(p.x, p.y, p.z, 0.0f);
            fvel[id - nb] = make_float4(v.x, v.y, v.z, 0.0f);
        }
    } else if (i < n + nb) {
        int b = i - n;
        float4 p = bpos[b], v = bvel[b];
        opos[b] = make_float4(p.x, p.y, p.z, 0.0f);
        ovel[b] = make_float4(v.x, v.y, v.z, 0.0f);
    }
}

// out[id(slot)] = field[slot] for 4-, 16-byte fields
template <class T>
__global__ void k_by_id(const float4* __restrict__ pos, const T* __restrict__ field, int n,
                        T* __restrict__ out)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[__float_as_int(pos[i].w)] = field[i];
}

// The velocity each boid's attached particle carries into the next step
// (its slot of the step's sorted order).
__global__ void k_att_vel(const float4* __restrict__ vel, const int* __restrict__ slot_of_boid, int nb,
                          float4* __restrict__ out)
{
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nb) out[b] = vel[slot_of_boid[b]];
}

__global__ void k_pressure_by_id(const float4* __restrict__ pos, const float* __restrict__ rho, Scenes sc,
                                 float* __restrict__ out)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < sc.n_all) {
        const StepConst& c = sc.c[scene_of(sc.pbase, sc.S, (unsigned)i)];
        out[__float_as_int(pos[i].w)] = c.k * (rho[i] - c.rho0);
    }
}

__global__ void k_ids(const float4* __restrict__ pos, int n, int* __restrict__ out)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = __float_as_int(pos[i].w);
}

// ------------------------------------------------------------------ API

extern "C" {

const char* sph_last_error(sph_handle* h) { return h ? h->msg : g_msg; }

long long sph_launch_count(sph_handle* h) { return h ? h->launches : 0; }

int sph_grid_dims(const sph_params* p, int which, int dims[3])
{
    if (!p || !dims || (which != 0 && which != 1)) return fail(nullptr, SPH_ERR_ARG, "bad arguments");
    GridDesc g;
    float d = which ? p->boid_cell_size : p->cell_size;
    if (!(d > 0.0f)) return fail(nullptr, SPH_ERR_ARG, "cell size must be > 0");
    if (make_grid_x(p->box_min, p->box_max, which ? d : cell_x(p), d, &g) != SPH_OK)
        return fail(nullptr, SPH_ERR_OVERFLOW, "grid too large");
    for (int a = 0; a < 3; ++a) dims[a] = g.dim[a];
    return SPH_OK;
}

int sph_lattice_mass(const sph_params* p, float spacing, float* mass)
{
    if (!p || !mass || !(spacing > 0.0f) || !(p->h > 0.0f) || !(p->rho0 > 0.0f))
        return fail(nullptr, SPH_ERR_ARG, "bad arguments");
    const double h = p->h, s = spacing, pi = 3.14159265358979323846;
    const int R = (int)ceil(h / s) + 1;
    double acc = 0.0;
    for (int z = -R; z <= R; ++z)
        for (int y = -R; y <= R; ++y)
            for (int x = -R; x <= R; ++x) {
                double r2 = (double)(x * x + y * y + z * z) * s * s;
                if (r2 < h * h) {
                    double t = h * h - r2;
                    acc += t * t * t;
                }
            }
    *mass = (float)((double)p->rho0 / (315.0 / (64.0 * pi * pow(h, 9)) * acc));
    return SPH_OK;
}

// Fill the host-side scene tables of h (S scenes) and the totals.
static int layout_scenes(sph_handle* h, const sph_params* params, const int* n_fluid, const int* n_boid, int S)
{
    if (S < 1 || !params || !n_fluid || !n_boid) return fail(nullptr, SPH_ERR_ARG, "need S >= 1 and the arrays");
    h->S = S;
    h->params = new (std::nothrow) sph_params[S];
    h->consts = new (std::nothrow) StepConst[S];
    h->h_pbase = new (std::nothrow) unsigned[S + 1];
    h->h_bbase = new (std::nothrow) unsigned[S + 1];
    if (!h->params || !h->consts || !h->h_pbase || !h->h_bbase) return fail(nullptr, SPH_ERR_ARG, "out of host memory");
    long long n = 0, nb = 0, nf = 0, C = 0, Cb = 0, Cf = 0;
    h->stats_chunks = 1;
    for (int k = 0; k < S; ++k) {
        int rc = validate(&params[k], n_fluid[k], n_boid[k]);
        if (rc != SPH_OK) return rc;
        h->params[k] = params[k];
        make_const(&params[k], n_fluid[k], n_boid[k], &h->consts[k]);
        h->h_pbase[k] = (unsigned)n;
        h->h_bbase[k] = (unsigned)nb;
        h->consts[k].p_base = (int)n;
        h->consts[k].b_base = (int)nb;
        h->consts[k].c_base = (int)C;
        h->consts[k].cb_base = (int)Cb;
        h->consts[k].fc_base = (int)Cf;
        Cf += (long long)h->consts[k].fdim[0] * h->consts[k].fdim[1] * h->consts[k].fdim[2];
        n += (long long)n_fluid[k] + n_boid[k];
        nb += n_boid[k];
        nf += n_fluid[k];
        C += h->consts[k].g.ncells;
        Cb += h->consts[k].gb.ncells;
        const long long span = std::max((long long)n_fluid[k] + n_boid[k], (long long)h->consts[k].g.ncells);
        h->stats_chunks = std::max(h->stats_chunks, (int)((span + STATS_CHUNK - 1) / STATS_CHUNK));
        if (n > 2147483647LL || C > 2147483646LL || Cb > 2147483646LL || Cf > 2147483646LL)
            return fail(nullptr, SPH_ERR_OVERFLOW, "the batch exceeds 2^31 particles or cells");
    }
    h->h_pbase[S] = (unsigned)n;
    h->h_bbase[S] = (unsigned)nb;
    for (int k = 0; k < S; ++k) h->consts[k].nb_all = (int)nb;
    h->n = (int)n;
    h->n_boid = (int)nb;
    h->n_fluid = (int)nf;
    h->ncells = (int)C;
    h->nbcells = (int)Cb;
    h->nfcells = (int)Cf;
    h->tune.block = 256;
    h->tune.use_seg = 1;
    h->tune.ppt = 1;
    h->tune.pipe_tile = 0;
    h->tune.pipe_block = 256;
    return SPH_OK;
}

static void free_tables(sph_handle* h)
{
    delete[] h->params;
    delete[] h->consts;
    delete[] h->h_pbase;
    delete[] h->h_bbase;
}

int sph_batch_workspace_size(const sph_params* params, const int* n_fluid, const int* n_boid, int S,
                             size_t* bytes)
{
    if (!bytes) return fail(nullptr, SPH_ERR_ARG, "bytes is NULL");
    sph_handle tmp;
    memset(&tmp, 0, sizeof(tmp));
    int rc = layout_scenes(&tmp, params, n_fluid, n_boid, S);
    if (rc == SPH_OK) *bytes = carve(&tmp, 0);
    free_tables(&tmp);
    return rc;
}

int sph_workspace_size(const sph_params* p, int n_fluid, int n_boid, size_t* bytes)
{
    return sph_batch_workspace_size(p, &n_fluid, &n_boid, 1, bytes);
}

int sph_batch_create(const sph_params* params, const int* n_fluid, const int* n_boid, int S, void* workspace,
                     size_t ws_bytes, sph_handle** out)
{
    if (!out) return fail(nullptr, SPH_ERR_ARG, "out is NULL");
    if (!workspace || ((uintptr_t)workspace & 255))
        return fail(nullptr, SPH_ERR_ARG, "workspace must be non-NULL and 256-byte aligned");
    sph_handle* h = new (std::nothrow) sph_handle;
    if (!h) return fail(nullptr, SPH_ERR_ARG, "out of host memory");
    memset(h, 0, sizeof(*h));
    int rc = layout_scenes(h, params, n_fluid, n_boid, S);
    if (rc != SPH_OK) {
        free_tables(h);
        delete h;
        return rc;
    }
    h->skip_cta = -1;
    size_t need = carve(h, (uintptr_t)workspace);
    if (ws_bytes < need) {
        free_tables(h);
        delete h;
        return fail(nullptr, SPH_ERR_ARG, "workspace too small: %zu < %zu bytes", ws_bytes, need);
    }
    cudaError_t e = cudaMemcpy(h->d_consts, h->consts, sizeof(StepConst) * (size_t)S, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(h->d_pbase, h->h_pbase, sizeof(unsigned) * (size_t)(S + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(h->d_bbase, h->h_bbase, sizeof(unsigned) * (size_t)(S + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(h->err, 0, 4 * sizeof(unsigned));
    if (e == cudaSuccess) e = prepare_kernels();
    if (e == cudaSuccess && h->n_boid > 0) {
        // default priority: a higher one lets the F_b warps take SMs from the
        // fluid blocks early and slows the force pass by more than it saves
        e = cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_dens, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        destroy_side(h);
        free_tables(h);
        delete h;
        return fail(nullptr, SPH_ERR_CUDA, "uploading the scene tables: %s", cudaGetErrorString(e));
    }
    h->sc.c = h->d_consts;
    h->sc.pbase = h->d_pbase;
    h->sc.bbase = h->d_bbase;
    h->sc.S = S;
    h->sc.n_all = h->n;
    h->sc.nb_all = h->n_boid;
    *out = h;
    return SPH_OK;
}

int sph_create(const sph_params* p, int n_fluid, int n_boid, void* workspace, size_t ws_bytes, sph_handle** out)
{
    return sph_batch_create(p, &n_fluid, &n_boid, 1, workspace, ws_bytes, out);
}

int sph_set_tuning(sph_handle* h, int block, int use_segments)
{
    if (!h) return fail(nullptr, SPH_ERR_ARG, "handle is NULL");
    if (block != 64 && block != 128 && block != 256 && block != 512)
        return fail(h, SPH_ERR_ARG, "block must be 64, 128, 256 or 512");
    if (use_segments != 0 && use_segments != 1) return fail(h, SPH_ERR_ARG, "use_segments must be 0 or 1");
    h->tune.block = block;
    h->tune.use_seg = use_segments;
    if (h->graph) {
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
    drop_boid_graphs(h);
    return SPH_OK;
}

int sph_set_particles_per_thread(sph_handle* h, int ppt)
{
    if (!h) return fail(nullptr, SPH_ERR_ARG, "handle is NULL");
    if (ppt != 1 && ppt != 2 && ppt != 4) return fail(h, SPH_ERR_ARG, "ppt must be 1, 2 or 4");
    h->tune.ppt = ppt;
    if (h->graph) {
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
    drop_boid_graphs(h);
    return SPH_OK;
}

int sph_set_pipeline(sph_handle* h, int tile_slots, int block)
{
    if (!h) return fail(nullptr, SPH_ERR_ARG, "handle is NULL");
    if (tile_slots != 0 && (tile_slots < 32 || tile_slots > 65536 || tile_slots % 32))
        return fail(h, SPH_ERR_ARG, "tile_slots must be 0 or a multiple of 32 in [32, 65536]");
    if (block != 128 && block != 256) return fail(h, SPH_ERR_ARG, "block must be 128 or 256");
    h->tune.pipe_tile = tile_slots;
    h->tune.pipe_block = block;
    if (h->graph) {
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
    return SPH_OK;
}

int sph_debug_barrier_skip(sph_handle* h, int cta)
{
    if (!h) return fail(nullptr, SPH_ERR_ARG, "handle is NULL");
    if (cta < -1) return fail(h, SPH_ERR_ARG, "cta must be >= -1");
    h->skip_cta = cta;
    if (h->graph) {
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
    return SPH_OK;
}

int sph_set_diagnostics(sph_handle* h, int record)
{
    if (!h) return fail(nullptr, SPH_ERR_ARG, "handle is NULL");
    if (record != 0 && record != 1) return fail(h, SPH_ERR_ARG, "record must be 0 or 1");
    h->diag = record != 0;
    if (h->graph) {  // the captured step holds the old choice
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
    return SPH_OK;
}

static void prof_free(sph_handle* h)
{
    for (int i = 0; i < 2 * h->prof_cap; ++i) cudaEventDestroy(h->prof_ev[i]);
    free(h->prof_ev);
    free(h->prof_kind);
    h->prof_ev = nullptr;
    h->prof_kind = nullptr;
    h->prof_cap = h->prof_n = 0;
}

int sph_set_neighbor_lists(sph_handle* h, void* pair_buffer, size_t bytes)
{
    if (!h) return fail(nullptr, SPH_ERR_ARG, "handle is NULL");
    if (pair_buffer && ((uintptr_t)pair_buffer & 3)) return fail(h, SPH_ERR_ARG, "pair buffer must be 4-byte aligned");
    if (!pair_buffer || bytes < 4) {
        h->list = nullptr;
        h->list_cap = 0;
    } else {
        h->list = (unsigned*)pair_buffer;
        h->list_cap = bytes / 4;
    }
    if (h->graph) {  // the captured step no longer matches
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
    return SPH_OK;
}

void sph_destroy(sph_handle* h)
{
    if (!h) return;
    prof_free(h);
    if (h->graph) cudaGraphExecDestroy(h->graph);
    drop_boid_graphs(h);
    destroy_side(h);
    free_tables(h);
    delete h;
}

int sph_profile_enable(sph_handle* h, int max_passes)
{
    if (!h || max_passes < 0) return fail(h, SPH_ERR_ARG, "bad arguments");
    prof_free(h);
    if (max_passes == 0) return SPH_OK;
    h->prof_ev = (cudaEvent_t*)calloc((size_t)max_passes * 2, sizeof(cudaEvent_t));
    h->prof_kind = (int*)calloc((size_t)max_passes, sizeof(int));
    if (!h->prof_ev || !h->prof_kind) {
        prof_free(h);
        return fail(h, SPH_ERR_ARG, "out of host memory");
    }
    for (int i = 0; i < 2 * max_passes; ++i) {
        cudaError_t e = cudaEventCreate(&h->prof_ev[i]);
        if (e != cudaSuccess) {
            h->prof_cap = i / 2;
            prof_free(h);
            return fail(h, SPH_ERR_CUDA, "cudaEventCreate: %s", cudaGetErrorString(e));
        }
        h->prof_cap = (i + 1) / 2;
    }
    h->prof_cap = max_passes;
    h->prof_n = 0;
    return SPH_OK;
}

int sph_profile_read(sph_handle* h, double* ms, long long* passes, int nkinds)
{
    if (!h || !ms || !passes || nkinds < 0) return fail(h, SPH_ERR_ARG, "bad arguments");
    for (int k = 0; k < nkinds; ++k) {
        ms[k] = 0.0;
        passes[k] = 0;
    }
    for (int i = 0; i < h->prof_n; ++i) {
        float t = 0.0f;
        // passes on the side stream may end after later passes of the caller's stream
        CUDA_TRY(h, cudaEventSynchronize(h->prof_ev[2 * i + 1]));
        CUDA_TRY(h, cudaEventElapsedTime(&t, h->prof_ev[2 * i], h->prof_ev[2 * i + 1]));
        int k = h->prof_kind[i];
        if (k < nkinds) {
            ms[k] += t;
            passes[k] += 1;
        }
    }
    h->prof_n = 0;
    return SPH_OK;
}

static bool aligned16(const void* ptr) { return ((uintptr_t)ptr & 15) == 0; }

int sph_set_state(sph_handle* h, const float* fluid_pos4, const float* fluid_vel4, const float* boid_pos4,
                  const float* boid_vel4, int on_host, void* stream)
{
    if (!h) return fail(nullptr, SPH_ERR_ARG, "handle is NULL");
    const int nf = h->n_fluid, nb = h->n_boid;
    if ((nf && (!fluid_pos4 || !fluid_vel4)) || (nb && (!boid_pos4 || !boid_vel4)))
        return fail(h, SPH_ERR_ARG, "state pointer is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    h->last_stream = s;
    const float4 *fp = (const float4*)fluid_pos4, *fv = (const float4*)fluid_vel4;
    const float4 *bp = (const float4*)boid_pos4, *bv = (const float4*)boid_vel4;
    if (on_host) {
        // stage in the sorted scratch arrays: fluid at [0, nf), boids at [nf, nf + nb)
        if (nf) {
            CUDA_TRY(h, cudaMemcpyAsync(h->pos_s, fluid_pos4, (size_t)nf * 16, cudaMemcpyHostToDevice, s));
            CUDA_TRY(h, cudaMemcpyAsync(h->vel_s, fluid_vel4, (size_t)nf * 16, cudaMemcpyHostToDevice, s));
        }
        if (nb) {
            CUDA_TRY(h, cudaMemcpyAsync(h->pos_s + nf, boid_pos4, (size_t)nb * 16, cudaMemcpyHostToDevice, s));
            CUDA_TRY(h, cudaMemcpyAsync(h->vel_s + nf, boid_vel4, (size_t)nb * 16, cudaMemcpyHostToDevice, s));
        }
        fp = h->pos_s;
        fv = h->vel_s;
        bp = h->pos_s + nf;
        bv = h->vel_s + nf;
    } else if (!aligned16(fp) || !aligned16(fv) || !aligned16(bp) || !aligned16(bv)) {
        return fail(h, SPH_ERR_ARG, "device state pointers must be 16-byte aligned");
    }
    if (h->n > 0) {
        k_load_state<<<(h->n + 255) / 256, 256, 0, s>>>(fp, fv, bp, bv, h->sc, h->pos, h->vel, h->bpos, h->bvel,
                                                         h->slot_of_boid);
        ++h->launches;
        CUDA_TRY(h, cudaGetLastError());
    }
    if (on_host) CUDA_TRY(h, cudaStreamSynchronize(s));
    h->has_state = true;
    h->keys_ready = false;
    h->has_step = false;
    return SPH_OK;
}

int sph_get_state(sph_handle* h, float* fluid_pos4, float* fluid_vel4, float* boid_pos4, float* boid_vel4,
                  int on_host, void* stream)
{
    if (!h) return fail(nullptr, SPH_ERR_ARG, "handle is NULL");
    if (!h->has_state) return fail(h, SPH_ERR_STATE, "no state loaded");
    const int nf = h->n_fluid, nb = h->n_boid;
    if ((nf && (!fluid_pos4 || !fluid_vel4)) || (nb && (!boid_pos4 || !boid_vel4)))
        return fail(h, SPH_ERR_ARG, "state pointer is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    h->last_stream = s;
    float4 *fp = (float4*)fluid_pos4, *fv = (float4*)fluid_vel4, *bp = (float4*)boid_pos4, *bv = (float4*)boid_vel4;
    if (on_host) {
        fp = h->pos_s;
        fv = h->vel_s;
        bp = h->pos_s + nf;
        bv = h->vel_s + nf;
    } else if (!aligned16(fp) || !aligned16(fv) || !aligned16(bp) || !aligned16(bv)) {
        return fail(h, SPH_ERR_ARG, "device state pointers must be 16-byte aligned");
    }
    if (h->n + nb > 0) {
        k_store_state<<<(h->n + nb + 255) / 256, 256, 0, s>>>(h->pos, h->vel, h->bpos, h->bvel, h->n, nb, fp, fv,
                                                               bp, bv);
        ++h->launches;
        CUDA_TRY(h, cudaGetLastError());
    }
    if (on_host) {
        if (nf) {
            CUDA_TRY(h, cudaMemcpyAsync(fluid_pos4, h->pos_s, (size_t)nf * 16, cudaMemcpyDeviceToHost, s));
            CUDA_TRY(h, cudaMemcpyAsync(fluid_vel4, h->vel_s, (size_t)nf * 16, cudaMemcpyDeviceToHost, s));
        }
        if (nb) {
            CUDA_TRY(h, cudaMemcpyAsync(boid_pos4, h->pos_s + nf, (size_t)nb * 16, cudaMemcpyDeviceToHost, s));
            CUDA_TRY(h, cudaMemcpyAsync(boid_vel4, h->vel_s + nf, (size_t)nb * 16, cudaMemcpyDeviceToHost, s));
        }
        CUDA_TRY(h, cudaStreamSynchronize(s));
        h->has_step = false;  // the scratch arrays held the staged copy
    }
    return SPH_OK;
}

static SoaPos soa_of(const sph_handle* h)
{
    const size_t st = soa_stride((size_t)h->n);
    return SoaPos{h->soa, h->soa + st, h->soa + 2 * st};
}

// Keys (if needed), scan, scatter and per-cell sort + gather of the state
// into the sorted scratch arrays.  consume = true zeroes the counts for the
// next step's keys.
static int bin_state(sph_handle* h, cudaStream_t s, bool consume)
{
    if (!h->keys_ready) {
        prof_begin(h, SPH_KIND_KEYS, s);
        CUDA_TRY(h, cudaMemsetAsync(h->count, 0, (size_t)h->ncells * sizeof(unsigned), s));
        CUDA_TRY(h, launch_scene_keys(h->pos, h->sc, h->key, h->rank, h->count, h->err, s, &h->launches));
        prof_end(h, s);
        h->keys_ready = true;
    }
    prof_begin(h, SPH_KIND_SCAN, s);
    CUDA_TRY(h, launch_scan(h->count, h->ncells, h->scan_part, h->cell_start, s, &h->launches));
    prof_end(h, s);
    prof_begin(h, SPH_KIND_SCATTER, s);
    CUDA_TRY(h, launch_scatter_ids(h->key, h->rank, h->cell_start, h->pos, h->n, h->tmp, h->tmp_id, s,
                                   &h->launches));
    prof_end(h, s);
    prof_begin(h, SPH_KIND_SORT, s);
    CUDA_TRY(h, launch_cellsort_slots(h->cell_start, h->key, h->n, h->ncells, h->tmp, h->tmp_id, h->pos, h->vel,
                                      h->pos_s, h->vel_s, h->soa, h->n_boid, h->slot_of_boid, h->big_list,
                                      h->big_count, s, &h->launches));
    prof_end(h, s);
    if (consume) {
        CUDA_TRY(h, cudaMemsetAsync(h->count, 0, (size_t)h->ncells * sizeof(unsigned), s));
        h->keys_ready = false;
    }
    return SPH_OK;
}

// The boids' binning (the boid state only) on stream s.
static int enqueue_boid_bin(sph_handle* h, cudaStream_t s)
{
    prof_begin(h, SPH_KIND_BOID_BIN, s);
    CUDA_TRY(h, cudaMemsetAsync(h->bcount, 0, (size_t)h->nbcells * sizeof(unsigned), s));
    CUDA_TRY(h, launch_boid_keys(h->bpos, h->sc, h->bkey, h->brank, h->bcount, s, &h->launches));
    CUDA_TRY(h, launch_scan(h->bcount, h->nbcells, h->bscan_part, h->bstart, s, &h->launches));
    CUDA_TRY(h, launch_scatter(h->bkey, h->brank, h->bstart, h->n_boid, h->btmp, s, &h->launches));
    CUDA_TRY(h, launch_cellsort_gather(h->bstart, h->nbcells, h->btmp, h->bpos, h->bvel, h->bpos_s, h->bvel_s, 0,
                                       nullptr, h->bbig_list, h->bbig_count, s, &h->launches));
    prof_end(h, s);
    return SPH_OK;
}

// The boid rules (needs F_b and the boids' binning) on stream s.
static cudaError_t launch_rules(sph_handle* h, cudaStream_t s)
{
    return launch_boid_rules(h->bpos_s, h->bvel_s, h->bstart, h->obst, h->sc, h->fb, h->vel_s, h->bpos, h->bvel,
                             h->pos, h->vel, h->slot_of_boid, h->key, h->rank, h->count, h->err, s, &h->launches);
}

// The density pass, the neighbour lists (when set) and the force pass as
// separate launches.  split: the F_b warps and the boid rules run on the
// side stream once the densities exist, alongside the fluid blocks of the
// force pass on s (they write disjoint slots: the fluid blocks write the
// fluid particles' next state and keys, the boid rules the boids' and their
// attached particles'; both only add to the cell counts), and s waits for
// them before it goes on.
static int enqueue_neighbor_passes(sph_handle* h, cudaStream_t s, bool split)
{
    prof_begin(h, SPH_KIND_DENSITY, s);
    CUDA_TRY(h, launch_density(h->pos_s, h->vel_s, soa_of(h), h->cell_start, h->sc, h->tune, h->rho, h->ab, h->prec,
                               h->nbr, h->seg, h->nseg, h->ncand, nullptr, nullptr, h->err, s, &h->launches));
    prof_end(h, s);
    if (h->list) {
        prof_begin(h, SPH_KIND_LISTS, s);
        CUDA_TRY(h, launch_scan((const unsigned*)h->nbr, h->n, h->noff_part, h->noff, s, &h->launches));
        CUDA_TRY(h, launch_fill_lists(h->pos_s, h->cell_start, h->sc, h->noff, h->list, h->list_cap, h->err, s,
                                      &h->launches));
        prof_end(h, s);
    }
    if (split) {
        CUDA_TRY(h, cudaEventRecord(h->ev_dens, s));
        CUDA_TRY(h, cudaStreamWaitEvent(h->side, h->ev_dens, 0));
        prof_begin(h, SPH_KIND_BOID_RULES, h->side);
        CUDA_TRY(h, launch_forces(h->pos_s, soa_of(h), h->vel_s, h->rho, h->ab, h->prec, h->cell_start, h->seg,
                                  h->nseg, h->sc, h->tune, h->list, h->noff, h->list_cap, true, false,
                                  h->slot_of_boid, nullptr, h->fb, h->diag ? h->acc : nullptr, nullptr, nullptr,
                                  h->pos, h->vel, h->key, h->rank, h->count, h->err, h->side, &h->launches));
        CUDA_TRY(h, launch_rules(h, h->side));
        prof_end(h, h->side);
        CUDA_TRY(h, cudaEventRecord(h->ev_join, h->side));
    }
    prof_begin(h, SPH_KIND_FORCES, s);
    CUDA_TRY(h, launch_forces(h->pos_s, soa_of(h), h->vel_s, h->rho, h->ab, h->prec, h->cell_start, h->seg, h->nseg, h->sc,
                              h->tune, h->list, h->noff, h->list_cap, !split, true, h->slot_of_boid, nullptr, h->fb,
                              h->diag ? h->acc : nullptr, h->diag ? h->touched : nullptr,
                              h->diag ? h->infl : nullptr, h->pos, h->vel, h->key, h->rank, h->count, h->err, s,
                              &h->launches));
    prof_end(h, s);
    if (split) CUDA_TRY(h, cudaStreamWaitEvent(s, h->ev_join, 0));
    return SPH_OK;
}

// Enqueue one step (keys must be ready or are computed first).  With boids
// and separate neighbour-pass launches, the boids' binning, F_b and rules
// run on the side stream, forked from s at the start of the step and joined
// back before it ends; the per-thread arithmetic is that of the serial order.
static int enqueue_step(sph_handle* h, cudaStream_t s)
{
    const bool pipe = h->tune.pipe_tile > 0 && !h->list;
    const bool split = h->n_boid > 0 && h->side && !pipe;
    if (split) {
        CUDA_TRY(h, cudaEventRecord(h->ev_fork, s));
        CUDA_TRY(h, cudaStreamWaitEvent(h->side, h->ev_fork, 0));
        int rc = enqueue_boid_bin(h, h->side);
        if (rc != SPH_OK) return rc;
    }
    int rc = bin_state(h, s, true);
    if (rc != SPH_OK) return rc;
    if (pipe) {
        // both neighbour passes in one cooperative launch
        prof_begin(h, SPH_KIND_PIPELINE, s);
        CUDA_TRY(h, launch_nbr_pipeline(h->pos_s, soa_of(h), h->vel_s, h->cell_start, h->sc, h->tune, h->rho, h->ab,
                                        h->prec, h->nbr, h->seg, h->nseg, h->ncand, h->slot_of_boid, h->fb,
                                        h->diag ? h->acc : nullptr, h->diag ? h->touched : nullptr,
                                        h->diag ? h->infl : nullptr, h->pos, h->vel, h->key, h->rank, h->count,
                                        h->pipe_queue, h->skip_cta, h->err, s, &h->launches));
        prof_end(h, s);
    } else {
        int rc2 = enqueue_neighbor_passes(h, s, split);
        if (rc2 != SPH_OK) return rc2;
    }
    if (h->n_boid > 0 && !split) {
        rc = enqueue_boid_bin(h, s);
        if (rc != SPH_OK) return rc;
        prof_begin(h, SPH_KIND_BOID_RULES, s);
        CUDA_TRY(h, launch_rules(h, s));
        prof_end(h, s);
    }
    h->keys_ready = true;  // the force and boid kernels emitted the next keys
    h->has_step = true;
    h->diag_step = h->diag;
    return SPH_OK;
}

int sph_step(sph_handle* h, int nsteps, void* stream)
{
    if (!h) return fail(nullptr, SPH_ERR_ARG, "handle is NULL");
    if (nsteps < 0) return fail(h, SPH_ERR_ARG, "nsteps < 0");
    if (!h->has_state) return fail(h, SPH_ERR_STATE, "no state loaded");
    cudaStream_t s = (cudaStream_t)stream;
    h->last_stream = s;
    for (int it = 0; it < nsteps; ++it) {
        int rc = enqueue_step(h, s);
        if (rc != SPH_OK) return rc;
    }
    return SPH_OK;
}

int sph_graph_step(sph_handle* h, int nsteps, void* stream)
{
    if (!h) return fail(nullptr, SPH_ERR_ARG, "handle is NULL");
    if (nsteps < 0) return fail(h, SPH_ERR_ARG, "nsteps < 0");
    if (!stream) return fail(h, SPH_ERR_ARG, "a CUDA graph needs a non-default stream");
    if (!h->has_state) return fail(h, SPH_ERR_STATE, "no state loaded");
    cudaStream_t s = (cudaStream_t)stream;
    h->last_stream = s;
    if (nsteps == 0) return SPH_OK;
    if (!h->keys_ready) {  // the captured step starts from emitted keys
        int rc = enqueue_step(h, s);
        if (rc != SPH_OK) return rc;
        --nsteps;
    }
    if (h->graph && h->graph_stream != s) {
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
    if (!h->graph && nsteps > 0) {
        const int cap = h->prof_cap;
        h->prof_cap = 0;  // no event records inside the graph
        const long long before = h->launches;
        cudaGraph_t g = nullptr;
        CUDA_TRY(h, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        int rc = enqueue_step(h, s);
        cudaError_t e = cudaStreamEndCapture(s, &g);
        h->prof_cap = cap;
        h->launches = before;
        if (rc != SPH_OK) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (e != cudaSuccess) return fail(h, SPH_ERR_CUDA, "stream capture: %s", cudaGetErrorString(e));
        size_t nodes = 0;
        cudaGraphGetNodes(g, nullptr, &nodes);
        e = cudaGraphInstantiate(&h->graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            h->graph = nullptr;
            return fail(h, SPH_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
        }
        h->graph_stream = s;
        h->graph_launches = (long long)nodes;
    }
    for (int it = 0; it < nsteps; ++it) {
        CUDA_TRY(h, cudaGraphLaunch(h->graph, s));
        h->launches += h->graph_launches;
    }
    h->keys_ready = true;
    h->has_step = true;
    h->diag_step = h->diag;
    return SPH_OK;
}

int sph_set_surrogate(sph_handle* h, sph_mlp* m, float f_scale, float log_err_max)
{
    if (!h) return fail(nullptr, SPH_ERR_ARG, "handle is NULL");
    if (m && !(isfinite(f_scale) && f_scale > 0.0f)) return fail(h, SPH_ERR_ARG, "f_scale must be > 0");
    h->mlp = m;
    h->f_scale = f_scale;
    h->log_err_max = log_err_max;
    drop_boid_graphs(h);  // the captured calls hold the old network and gate
    return SPH_OK;
}

int sph_set_surrogate_bounds(sph_handle* h, const float* lo, const float* hi)
{
    if (!h) return fail(nullptr, SPH_ERR_ARG, "handle is NULL");
    if ((lo == nullptr) != (hi == nullptr)) return fail(h, SPH_ERR_ARG, "give both lo and hi, or neither");
    h->feat_lo = lo;
    h->feat_hi = hi;
    drop_boid_graphs(h);  // the captured calls hold the old range
    return SPH_OK;
}

int sph_features(sph_handle* h, void* x_out, void* stream)
{
    if (!h) return fail(nullptr, SPH_ERR_ARG, "handle is NULL");
    if (!h->has_state) return fail(h, SPH_ERR_STATE, "no state loaded");
    if (h->n_boid && (!x_out || !aligned16(x_out))) return fail(h, SPH_ERR_ARG, "x_out must be 16-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    h->last_stream = s;
    if (h->n_boid == 0) return SPH_OK;
    int rc = bin_state(h, s, false);
    if (rc != SPH_OK) return rc;
    prof_begin(h, SPH_KIND_FEATURES, s);
    CUDA_TRY(h, launch_features(h->pos_s, h->vel_s, h->cell_start, h->bpos, h->bvel, h->sc, h->fgrid, h->nfcells,
                                x_out, s, &h->launches));
    prof_end(h, s);
    h->has_step = false;
    return SPH_OK;
}

// Exact fluid force on the boids flagged in bmask (NULL: every boid),
// computing densities only where those forces need them.
// F_b of the boids in bmask (NULL: all) from the densities of only the
// particles they need: mark them, compact their slots into a list, run the
// density pass over the list and the force pass over the boids.
static int exact_local(sph_handle* h, const int* bmask, float4* out, cudaStream_t s)
{
    CUDA_TRY(h, cudaMemsetAsync(h->need, 0, (size_t)h->n, s));
    CUDA_TRY(h, launch_mark_needed(h->pos_s, h->cell_start, h->sc, h->slot_of_boid, bmask, h->need, s, &h->launches));
    CUDA_TRY(h, launch_compact_needed(h->need, h->n, h->need_list, h->need_len, s, &h->launches));
    CUDA_TRY(h, launch_density(h->pos_s, h->vel_s, soa_of(h), h->cell_start, h->sc, h->tune, h->rho, h->ab, nullptr,
                               h->nbr, nullptr, nullptr, h->ncand, h->need_list, h->need_len, h->err, s,
                               &h->launches));
    CUDA_TRY(h, launch_forces(h->pos_s, soa_of(h), h->vel_s, h->rho, h->ab, nullptr, h->cell_start, nullptr, nullptr,
                              h->sc, h->tune,
                              nullptr, nullptr, 0, true, false, h->slot_of_boid, bmask, out, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                              nullptr, nullptr, h->err, s, &h->launches));
    return SPH_OK;
}

// The launches of one sph_boid_forces call (arguments checked).
static int enqueue_boid_forces(sph_handle* h, int mode, float* out_f4, cudaStream_t s)
{
    int rc = bin_state(h, s, false);
    if (rc != SPH_OK) return rc;
    float4* out = (float4*)out_f4;
    h->has_step = false;
    if (mode == SPH_BOID_EXACT) {
        CUDA_TRY(h, launch_density(h->pos_s, h->vel_s, soa_of(h), h->cell_start, h->sc, h->tune, h->rho, h->ab,
                                   nullptr, h->nbr, nullptr, nullptr, h->ncand, nullptr, nullptr, h->err, s,
                                   &h->launches));
        CUDA_TRY(h, launch_forces(h->pos_s, soa_of(h), h->vel_s, h->rho, h->ab, nullptr, h->cell_start, nullptr,
                                  nullptr, h->sc, h->tune,
                                  nullptr, nullptr, 0, true, false, h->slot_of_boid, nullptr, out, nullptr, nullptr, nullptr, nullptr, nullptr,
                                  nullptr, nullptr, nullptr, h->err, s, &h->launches));
        return SPH_OK;
    }
    if (mode == SPH_BOID_EXACT_LOCAL) return exact_local(h, nullptr, out, s);
    // surrogate: features -> network -> forces (+ exact path for flagged boids)
    prof_begin(h, SPH_KIND_FEATURES, s);
    CUDA_TRY(h, launch_features(h->pos_s, h->vel_s, h->cell_start, h->bpos, h->bvel, h->sc, h->fgrid, h->nfcells,
                                h->feat, s, &h->launches));
    prof_end(h, s);
    rc = sph_mlp_forward(h->mlp, h->feat, h->nb_pad, h->yout, s);
    if (rc != SPH_OK) return fail(h, rc, "surrogate forward: %s", sph_last_error(nullptr));
    CUDA_TRY(h, launch_surrogate_out(h->yout, h->feat, h->feat_lo, h->feat_hi, h->n_boid, h->f_scale, h->log_err_max,
                                     out, h->bflag, h->err + 1, s, &h->launches));
    if (mode == SPH_BOID_SURROGATE_FALLBACK) return exact_local(h, h->bflag, out, s);
    return SPH_OK;
}

static int check_boid_forces(sph_handle* h, int mode, float* out_f4)
{
    if (!h) return fail(nullptr, SPH_ERR_ARG, "handle is NULL");
    if (mode < SPH_BOID_EXACT || mode > SPH_BOID_EXACT_LOCAL) return fail(h, SPH_ERR_ARG, "unsupported mode %d", mode);
    if (h->n_boid && (!out_f4 || !aligned16(out_f4))) return fail(h, SPH_ERR_ARG, "out must be 16-byte aligned");
    if (!h->has_state) return fail(h, SPH_ERR_STATE, "no state loaded");
    if ((mode == SPH_BOID_SURROGATE || mode == SPH_BOID_SURROGATE_FALLBACK) && !h->mlp)
        return fail(h, SPH_ERR_STATE, "no surrogate attached (sph_set_surrogate)");
    return SPH_OK;
}

int sph_boid_forces(sph_handle* h, int mode, float* out_f4, void* stream)
{
    int rc = check_boid_forces(h, mode, out_f4);
    if (rc != SPH_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    h->last_stream = s;
    if (h->n_boid == 0) return SPH_OK;
    return enqueue_boid_forces(h, mode, out_f4, s);
}

int sph_graph_boid_forces(sph_handle* h, int mode, float* out_f4, void* stream)
{
    int rc = check_boid_forces(h, mode, out_f4);
    if (rc != SPH_OK) return rc;
    if (!stream) return fail(h, SPH_ERR_ARG, "a CUDA graph needs a non-default stream");
    cudaStream_t s = (cudaStream_t)stream;
    h->last_stream = s;
    if (h->n_boid == 0) return SPH_OK;
    auto& g = h->bgraph[mode - SPH_BOID_EXACT];
    if (g.exec && (g.out != out_f4 || g.stream != s)) {
        cudaGraphExecDestroy(g.exec);
        g.exec = nullptr;
    }
    if (!g.exec && (!g.warm || !h->keys_ready)) {
        // a plain call: the first of this mode (one-time set-up of its
        // kernels), or the state's cell keys are not computed yet
        rc = enqueue_boid_forces(h, mode, out_f4, s);
        if (rc == SPH_OK) g.warm = true;
        return rc;
    }
    if (!g.exec) {
        const int cap = h->prof_cap;
        h->prof_cap = 0;  // no event records inside the graph
        const long long before = h->launches;
        cudaGraph_t graph = nullptr;
        CUDA_TRY(h, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        rc = enqueue_boid_forces(h, mode, out_f4, s);
        cudaError_t e = cudaStreamEndCapture(s, &graph);
        h->prof_cap = cap;
        g.launches = h->launches - before;
        h->launches = before;
        if (rc != SPH_OK) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        if (e != cudaSuccess) return fail(h, SPH_ERR_CUDA, "stream capture: %s", cudaGetErrorString(e));
        e = cudaGraphInstantiate(&g.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            g.exec = nullptr;
            return fail(h, SPH_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
        }
        g.out = out_f4;
        g.stream = s;
    }
    if (!h->keys_ready) return enqueue_boid_forces(h, mode, out_f4, s);  // the captured call starts from keys
    CUDA_TRY(h, cudaGraphLaunch(g.exec, s));
    h->launches += g.launches;
    h->has_step = false;
    return SPH_OK;
}

int sph_debug_bucket_neighbors(sph_handle* h, void* scratch, size_t bytes, int capacity, int* counts,
                               unsigned long long* dropped, void* stream)
{
    if (!h) return fail(nullptr, SPH_ERR_ARG, "handle is NULL");
    if (!scratch || !counts || !dropped || capacity < 1) return fail(h, SPH_ERR_ARG, "bad arguments");
    if (((uintptr_t)scratch & 3) || ((uintptr_t)dropped & 7)) return fail(h, SPH_ERR_ARG, "misaligned buffers");
    const size_t need = (size_t)h->ncells * (1 + (size_t)capacity) * sizeof(unsigned);
    if (bytes < need) return fail(h, SPH_ERR_ARG, "scratch too small: %zu < %zu bytes", bytes, need);
    if (!h->has_state) return fail(h, SPH_ERR_STATE, "no state loaded");
    cudaStream_t s = (cudaStream_t)stream;
    h->last_stream = s;
    int rc = bin_state(h, s, false);
    if (rc != SPH_OK) return rc;
    unsigned* tracker = (unsigned*)scratch;
    CUDA_TRY(h, launch_bucket_neighbors(h->pos_s, h->cell_start, h->sc, tracker, (int)h->ncells, tracker + h->ncells,
                                        capacity, counts, dropped, s, &h->launches));
    h->has_step = false;
    return SPH_OK;
}

int sph_debug_neighbors(sph_handle* h, int* counts, const long long* offsets, int* list, void* stream)
{
    if (!h) return fail(nullptr, SPH_ERR_ARG, "handle is NULL");
    if (!counts || ((offsets == nullptr) != (list == nullptr)))
        return fail(h, SPH_ERR_ARG, "counts must be given; offsets and list together");
    if (!h->has_state) return fail(h, SPH_ERR_STATE, "no state loaded");
    cudaStream_t s = (cudaStream_t)stream;
    h->last_stream = s;
    int rc = bin_state(h, s, false);
    if (rc != SPH_OK) return rc;
    CUDA_TRY(h, launch_neighbor_list(h->pos_s, h->cell_start, h->sc, counts, offsets, list, s, &h->launches));
    h->has_step = false;
    return SPH_OK;
}

int sph_get_fields(sph_handle* h, int field, void* out, int on_host, void* stream)
{
    if (!h) return fail(nullptr, SPH_ERR_ARG, "handle is NULL");
    if (!out) return fail(h, SPH_ERR_ARG, "out is NULL");
    if (!h->has_step && field != SPH_FIELD_FALLBACK && field != SPH_FIELD_OBSTACLE_GRID)
        return fail(h, SPH_ERR_STATE, "no step since the state was loaded or staged");
    cudaStream_t s = (cudaStream_t)stream;
    h->last_stream = s;
    const int n = h->n, nb = h->n_boid;
    const int blocks = (n + 255) / 256;
    size_t bytes = 0;
    void* dst = on_host ? (void*)h->pos_s : out;  // staging: the sorted scratch array
    switch (field) {
    case SPH_FIELD_RHO:
        if (n) k_by_id<float><<<blocks, 256, 0, s>>>(h->pos, h->rho, n, (float*)dst);
        bytes = (size_t)n * 4;
        break;
    case SPH_FIELD_PRESSURE:
        if (n) k_pressure_by_id<<<blocks, 256, 0, s>>>(h->pos, h->rho, h->sc, (float*)dst);
        bytes = (size_t)n * 4;
        break;
    case SPH_FIELD_ACC:
        if (!h->diag_step) return fail(h, SPH_ERR_STATE, "acc is recorded only by steps taken with sph_set_diagnostics(h, 1)");
        if (n) k_by_id<float4><<<blocks, 256, 0, s>>>(h->pos, h->acc, n, (float4*)dst);
        bytes = (size_t)n * 16;
        break;
    case SPH_FIELD_TOUCHED:
        if (!h->diag_step) return fail(h, SPH_ERR_STATE, "touched is recorded only by steps taken with sph_set_diagnostics(h, 1)");
        if (n) k_by_id<int><<<blocks, 256, 0, s>>>(h->pos, h->touched, n, (int*)dst);
        bytes = (size_t)n * 4;
        break;
    case SPH_FIELD_INFLUENCE:
        if (!h->diag_step) return fail(h, SPH_ERR_STATE, "influence is recorded only by steps taken with sph_set_diagnostics(h, 1)");
        if (n) k_by_id<float4><<<blocks, 256, 0, s>>>(h->pos, h->infl, n, (float4*)dst);
        bytes = (size_t)n * 16;
        break;
    case SPH_FIELD_NBR_COUNT:
        if (n) k_by_id<int><<<blocks, 256, 0, s>>>(h->pos, h->nbr, n, (int*)dst);
        bytes = (size_t)n * 4;
        break;
    case SPH_FIELD_ATT_VEL:
        // the attached particle of boid b has id b: the first nb ids
        if (nb) k_att_vel<<<(nb + 255) / 256, 256, 0, s>>>(h->vel, h->slot_of_boid, nb, (float4*)dst);
        bytes = (size_t)nb * 16;
        break;
    case SPH_FIELD_OBSTACLE_GRID:
        bytes = (size_t)h->nbcells * 16;
        if (h->nbcells) CUDA_TRY(h, cudaMemcpyAsync(dst, h->obst, bytes, cudaMemcpyDeviceToDevice, s));
        break;
    case SPH_FIELD_FALLBACK:
        bytes = (size_t)nb * 4;
        if (nb) CUDA_TRY(h, cudaMemcpyAsync(dst, h->bflag, bytes, cudaMemcpyDeviceToDevice, s));
        break;
    case SPH_FIELD_NSEG:
        if (n) k_by_id<int><<<blocks, 256, 0, s>>>(h->pos, h->nseg, n, (int*)dst);
        bytes = (size_t)n * 4;
        break;
    case SPH_FIELD_NCAND:
        if (n) k_by_id<int><<<blocks, 256, 0, s>>>(h->pos, h->ncand, n, (int*)dst);
        bytes = (size_t)n * 4;
        break;
    case SPH_FIELD_KEYS:
        CUDA_TRY(h, launch_slot_keys(h->cell_start, h->ncells, (unsigned*)h->tmp, s, &h->launches));
        if (n) k_by_id<unsigned><<<blocks, 256, 0, s>>>(h->pos, (const unsigned*)h->tmp, n, (unsigned*)dst);
        bytes = (size_t)n * 4;
        break;
    case SPH_FIELD_PERM:
        if (n) k_ids<<<blocks, 256, 0, s>>>(h->pos, n, (int*)dst);
        bytes = (size_t)n * 4;
        break;
    case SPH_FIELD_CELL_START:
        dst = out;
        bytes = ((size_t)h->ncells + 1) * 4;
        CUDA_TRY(h, cudaMemcpyAsync(out, h->cell_start, bytes, on_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s));
        if (on_host) CUDA_TRY(h, cudaStreamSynchronize(s));
        return SPH_OK;
    case SPH_FIELD_FB:
        bytes = (size_t)nb * 16;
        if (nb) CUDA_TRY(h, cudaMemcpyAsync(dst, h->fb, bytes, cudaMemcpyDeviceToDevice, s));
        break;
    case SPH_FIELD_BOID_PERM:
        if (nb) k_ids<<<(nb + 255) / 256, 256, 0, s>>>(h->bpos_s, nb, (int*)dst);
        bytes = (size_t)nb * 4;
        break;
    case SPH_FIELD_BOID_KEYS:
        CUDA_TRY(h, launch_slot_keys(h->bstart, h->nbcells, (unsigned*)h->btmp, s, &h->launches));
        if (nb) k_by_id<unsigned><<<(nb + 255) / 256, 256, 0, s>>>(h->bpos_s, (const unsigned*)h->btmp, nb, (unsigned*)dst);
        bytes = (size_t)nb * 4;
        break;
    case SPH_FIELD_BOID_CELL_START:
        bytes = ((size_t)h->nbcells + 1) * 4;
        CUDA_TRY(h, cudaMemcpyAsync(out, h->bstart, bytes, on_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s));
        if (on_host) CUDA_TRY(h, cudaStreamSynchronize(s));
        return SPH_OK;
    default:
        return fail(h, SPH_ERR_ARG, "unknown field %d", field);
    }
    if (field != SPH_FIELD_FB && field != SPH_FIELD_FALLBACK && field != SPH_FIELD_KEYS &&
        field != SPH_FIELD_BOID_KEYS)
        ++h->launches;
    if (field == SPH_FIELD_KEYS || field == SPH_FIELD_BOID_KEYS) ++h->launches;
    CUDA_TRY(h, cudaGetLastError());
    if (on_host) {
        if (bytes) CUDA_TRY(h, cudaMemcpyAsync(out, dst, bytes, cudaMemcpyDeviceToHost, s));
        CUDA_TRY(h, cudaStreamSynchronize(s));
    }
    return SPH_OK;
}

int sph_stats(sph_handle* h, double* out, int on_host, void* stream)
{
    if (!h) return fail(nullptr, SPH_ERR_ARG, "handle is NULL");
    if (!out) return fail(h, SPH_ERR_ARG, "out is NULL");
    if (!h->has_step) return fail(h, SPH_ERR_STATE, "no step since the state was loaded or staged");
    cudaStream_t s = (cudaStream_t)stream;
    h->last_stream = s;
    const size_t bytes = (size_t)h->S * SPH_STATS_N * sizeof(double);
    double* dst = on_host ? h->stats_out : out;
    CUDA_TRY(h, launch_stats(h->pos, h->vel, h->rho, h->nbr, h->cell_start, h->sc, h->stats_chunks, h->stats_part,
                             dst, s, &h->launches));
    if (on_host) {
        CUDA_TRY(h, cudaMemcpyAsync(out, dst, bytes, cudaMemcpyDeviceToHost, s));
        CUDA_TRY(h, cudaStreamSynchronize(s));
    }
    return SPH_OK;
}

int sph_status(sph_handle* h, unsigned* bits)
{
    if (!h || !bits) return fail(h, SPH_ERR_ARG, "bad arguments");
    unsigned v = 0;
    CUDA_TRY(h, cudaMemcpyAsync(&v, h->err, sizeof(unsigned), cudaMemcpyDeviceToHost, h->last_stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->last_stream));
    *bits = v;
    return SPH_OK;
}

int sph_clear_status(sph_handle* h, void* stream)
{
    if (!h) return fail(nullptr, SPH_ERR_ARG, "handle is NULL");
    h->last_stream = (cudaStream_t)stream;
    CUDA_TRY(h, cudaMemsetAsync(h->err, 0, sizeof(unsigned), (cudaStream_t)stream));
    return SPH_OK;
}

}  // extern "C"

// ------------------------------------------------------------ surface

int sph_voxel_grid(const sph_params* p, float spacing, float radius, float* origin, int* dims)
{
    if (!p || !origin || !dims) return fail(nullptr, SPH_ERR_ARG, "NULL argument");
    if (!finite_pos(spacing) || !finite_pos(radius)) return fail(nullptr, SPH_ERR_ARG, "spacing and radius must be > 0");
    const int pad = (int)ceilf(radius / spacing) + 1;
    long long total = 1;
    for (int a = 0; a < 3; ++a) {
        const float ext = p->box_max[a] - p->box_min[a];
        if (!(ext > 0.0f) || !isfinite(ext)) return fail(nullptr, SPH_ERR_ARG, "empty box");
        const double n = floor((double)ext / spacing) + 1.0 + 2.0 * pad;
        if (n > 2147483647.0) return fail(nullptr, SPH_ERR_OVERFLOW, "too many corners");
        dims[a] = (int)n;
        origin[a] = p->box_min[a] - (float)pad * spacing;
        total *= dims[a];
    }
    if (total > 2147483647LL) return fail(nullptr, SPH_ERR_OVERFLOW, "more than 2^31 - 1 corners");
    return SPH_OK;
}

int sph_voxel_density(sph_handle* h, const float* origin, const int* dims, float spacing, float radius,
                      float particle_radius, float* phi, int* counts, void* stream)
{
    if (!h) return fail(nullptr, SPH_ERR_ARG, "handle is NULL");
    if (h->S != 1) return fail(h, SPH_ERR_ARG, "voxel density needs a single-scene handle");
    if (!origin || !dims || !phi) return fail(h, SPH_ERR_ARG, "NULL argument");
    if (((uintptr_t)phi & 3) || ((uintptr_t)counts & 3)) return fail(h, SPH_ERR_ARG, "misaligned output");
    if (!finite_pos(spacing) || !finite_pos(radius) || !(particle_radius >= 0.0f) || !isfinite(particle_radius))
        return fail(h, SPH_ERR_ARG, "spacing, radius must be > 0, particle_radius >= 0");
    long long total = 1;
    for (int a = 0; a < 3; ++a) {
        if (dims[a] < 1 || !isfinite(origin[a])) return fail(h, SPH_ERR_ARG, "bad grid");
        total *= dims[a];
    }
    if (total > 2147483647LL) return fail(h, SPH_ERR_OVERFLOW, "more than 2^31 - 1 corners");
    if (!h->has_state) return fail(h, SPH_ERR_STATE, "no state loaded");
    cudaStream_t s = (cudaStream_t)stream;
    h->last_stream = s;
    int rc = bin_state(h, s, false);
    if (rc != SPH_OK) return rc;
    VoxelConst v;
    for (int a = 0; a < 3; ++a) {
        v.dims[a] = dims[a];
        v.origin[a] = origin[a];
    }
    v.spacing = spacing;
    v.R = radius;
    v.R2 = radius * radius;
    v.invR2 = (float)(1.0 / (double)v.R2);
    v.r = particle_radius;
    v.wb = make_bounds(&h->params[0], v.R2, h->params[0].cell_size, cell_x(&h->params[0]));
    CUDA_TRY(h, launch_voxel_density(h->pos_s, h->cell_start, h->sc, v, phi, counts, s, &h->launches));
    h->has_step = false;
    return SPH_OK;
}

struct McLayout {
    long long ncubes;
    size_t tile_off, tile_count, count, cases, total;
};

static int mc_layout(const int* dims, McLayout* L)
{
    if (!dims || dims[0] < 1 || dims[1] < 1 || dims[2] < 1) return SPH_ERR_ARG;
    const long long n = (long long)(dims[0] - 1) * (dims[1] - 1) * (dims[2] - 1);
    if ((long long)dims[0] * dims[1] * dims[2] > 2147483647LL || n > 2147483647LL / 5) return SPH_ERR_OVERFLOW;
    L->ncubes = n;
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t nt = (size_t)(n > 0 ? mc_tiles(n) : 1);
    L->tile_off = 0;
    L->tile_count = up(nt * sizeof(unsigned long long));
    L->count = L->tile_count + up(nt * sizeof(unsigned));
    L->cases = L->count + 256;
    L->total = L->cases + up((size_t)(n > 0 ? n : 1));
    return SPH_OK;
}

int sph_mc_workspace_size(const int* dims, size_t* bytes)
{
    if (!bytes) return fail(nullptr, SPH_ERR_ARG, "NULL argument");
    McLayout L;
    const int rc = mc_layout(dims, &L);
    if (rc != SPH_OK) return fail(nullptr, rc, "bad or too large corner grid");
    *bytes = L.total;
    return SPH_OK;
}

int sph_marching_cubes(const float* phi, const int* dims, const float* origin, float spacing, float iso,
                       void* workspace, size_t ws_bytes, float* tris, long long max_tris, unsigned* ntri,
                       void* stream)
{
    if (!phi || !origin || !workspace || !ntri || (max_tris > 0 && !tris) || max_tris < 0)
        return fail(nullptr, SPH_ERR_ARG, "NULL argument or negative capacity");
    if (((uintptr_t)phi & 3) || ((uintptr_t)workspace & 255) || ((uintptr_t)tris & 3) || ((uintptr_t)ntri & 3))
        return fail(nullptr, SPH_ERR_ARG, "misaligned buffer (workspace: 256 bytes, others: 4)");
    if (!finite_pos(spacing) || !isfinite(iso)) return fail(nullptr, SPH_ERR_ARG, "spacing must be > 0, iso finite");
    for (int a = 0; a < 3; ++a)
        if (!isfinite(origin[a])) return fail(nullptr, SPH_ERR_ARG, "origin not finite");
    McLayout L;
    int rc = mc_layout(dims, &L);
    if (rc != SPH_OK) return fail(nullptr, rc, "bad or too large corner grid");
    if (ws_bytes < L.total) return fail(nullptr, SPH_ERR_ARG, "workspace too small: %zu < %zu bytes", ws_bytes, L.total);
    cudaError_t e = mc_upload_tables();
    if (e != cudaSuccess) return fail(nullptr, SPH_ERR_CUDA, "marching-cubes tables: %s", cudaGetErrorString(e));
    cudaStream_t s = (cudaStream_t)stream;
    uint8_t* w = (uint8_t*)workspace;
    unsigned* count = (unsigned*)(w + L.count);
    long long launches = 0;
    e = launch_marching_cubes(phi, dims, origin, spacing, iso, (unsigned char*)(w + L.cases), (unsigned*)(w + L.tile_count),
                              (unsigned long long*)(w + L.tile_off), count, tris, (unsigned long long)max_tris, s,
                              &launches);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ntri, count, sizeof(unsigned), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return fail(nullptr, SPH_ERR_CUDA, "marching cubes: %s", cudaGetErrorString(e));
    return SPH_OK;
}

int sph_mc_tables(unsigned short* edge_table, signed char* tri_table)
{
    if (mc_tables_host(edge_table, tri_table) != 0)
        return fail(nullptr, SPH_ERR_CUDA, "marching-cubes table generator failed its checks");
    return SPH_OK;
}

// ----------------------------------------------------------- obstacles

int sph_set_obstacles(sph_handle* h, const float* spheres, int n_sphere, const float* boxes, int n_box,
                      float w_obst, float near_factor, void* stream)
{
    if (!h) return fail(nullptr, SPH_ERR_ARG, "handle is NULL");
    if (h->S != 1) return fail(h, SPH_ERR_ARG, "obstacles need a single-scene handle");
    if (n_sphere < 0 || n_box < 0 || n_sphere + n_box > SPH_MAX_OBSTACLES)
        return fail(h, SPH_ERR_ARG, "0 <= n_sphere + n_box <= %d", SPH_MAX_OBSTACLES);
    if ((n_sphere && !spheres) || (n_box && !boxes)) return fail(h, SPH_ERR_ARG, "NULL obstacle array");
    if (!isfinite(w_obst) || !(near_factor >= 0.0f) || !isfinite(near_factor))
        return fail(h, SPH_ERR_ARG, "w_obst must be finite, near_factor >= 0");
    for (int k = 0; k < 4 * n_sphere; ++k)
        if (!isfinite(spheres[k]) || (k % 4 == 3 && !(spheres[k] > 0.0f)))
            return fail(h, SPH_ERR_ARG, "sphere %d: non-finite value or radius <= 0", k / 4);
    for (int k = 0; k < 6 * n_box; ++k)
        if (!isfinite(boxes[k]) || (k % 6 >= 3 && !(boxes[k] >= boxes[k - 3])))
            return fail(h, SPH_ERR_ARG, "box %d: non-finite value or max < min", k / 6);
    cudaStream_t s = (cudaStream_t)stream;
    h->last_stream = s;
    StepConst& c = h->consts[0];
    const int n = n_sphere + n_box;
    if (n > 0) {
        CUDA_TRY(h, cudaMemcpyAsync(h->obst_shapes, spheres, sizeof(float) * 4 * (size_t)n_sphere,
                                    cudaMemcpyHostToDevice, s));
        if (n_box)
            CUDA_TRY(h, cudaMemcpyAsync(h->obst_shapes + 4 * n_sphere, boxes, sizeof(float) * 6 * (size_t)n_box,
                                        cudaMemcpyHostToDevice, s));
        const float half_diag = 0.866025403784f * h->params[0].boid_cell_size;
        CUDA_TRY(h, launch_obstacle_grid(c, h->obst_shapes, n_sphere, n_box, half_diag, h->obst, s, &h->launches));
    } else if (h->nbcells) {
        CUDA_TRY(h, cudaMemsetAsync(h->obst, 0, (size_t)h->nbcells * sizeof(float4), s));
    }
    c.obst_on = n > 0 ? 1 : 0;
    c.obst_reach = (int)ceilf(h->params[0].r_vis / h->params[0].boid_cell_size) + 1;
    c.w_obst = w_obst;
    c.obst_near = near_factor;
    CUDA_TRY(h, cudaMemcpyAsync(h->d_consts, h->consts, sizeof(StepConst), cudaMemcpyHostToDevice, s));
    // the host copy must outlive the asynchronous copy: wait for it here
    CUDA_TRY(h, cudaStreamSynchronize(s));
    return SPH_OK;
}
