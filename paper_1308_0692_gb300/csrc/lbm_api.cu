// C-ABI of liblbm.so (declarations and contracts in include/lbm.h).
//
// Host side of the march: velocity-set construction, coefficients of the fully
// discrete scheme (time step from the CFL number, upwind Courant numbers, relaxation
// factor, wall-ghost coefficients of Eqs. 8-9), device memory layout, and the
// stream-ordered launch sequence of the fused step kernels.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_internal.h"

cudaError_t launch_step_f64_small(int m, int g, int pf, bool resid, const StepArgs &a, int grid, cudaStream_t s);
cudaError_t launch_step_f64_large(int m, int g, int pf, bool resid, const StepArgs &a, int grid, cudaStream_t s);
cudaError_t launch_step_f32_small(int m, int g, int pf, bool resid, const StepArgs &a, int grid, cudaStream_t s);
cudaError_t launch_step_f32_large(int m, int g, int pf, bool resid, const StepArgs &a, int grid, cudaStream_t s);
cudaError_t launch_defect_f32(int m, const StepArgs &a, int grid, cudaStream_t s);
cudaError_t launch_step_f32_tma(int m, int g, bool resid, const StepArgs &a, int grid, cudaStream_t s,
                               bool merged);
cudaError_t prepare_step_f32_tma(int m, int g);
cudaError_t launch_step_f32_march(int m, int g, int slots, bool defer, int tiled, bool resid, const StepArgs &a, int grid,
                                  cudaStream_t s);
cudaError_t prepare_step_f32_march(int m, int g, int slots, bool defer, int tiled, int *grid);
cudaError_t launch_step_so(int prec, int m, int g, bool resid, const StepArgs &a, int grid, cudaStream_t s);
bool so_supported(int prec, int m, int g);
cudaError_t launch_step_f32_so_march(int m, int g, int slots, int tiled, bool resid, const StepArgs &a, int grid,
                                     cudaStream_t s);
cudaError_t prepare_step_f32_so_march(int m, int g, int slots, int tiled, int *grid);
bool so_march_supported(int m, int g, int slots, int tiled);
// second-order transport on the strip-tiled state: load path 8 a ring of five row slots with
// direct stores, 9 a ring of four with bulk asynchronous stores (step_so_march.cu)
static int so_march_slots(int pf) { return pf == 8 ? 5 : 4; }
static int so_march_tiled(int pf) { return pf == 8 ? 1 : 2; }
bool march_supported(int m, int g, int slots, bool defer, int tiled);
int defect_lanes(int m);
int correct_lanes(int m);
cudaError_t launch_correct_f32(int m, int g, bool resid, const StepArgs &a, int grid,
                               cudaStream_t s);

struct lbm_vset {
    int kind;
    int n_arg;
    int m;
    std::vector<double> nodes, weights;   // 1-D rule, ascending
    std::vector<double> xi_x, xi_y, w;    // 2-D tensor product, a = iy*M + ix
};

struct lbm_sim {
    lbm_vset vs;
    lbm_problem prob;
    int nv;
    long ncells;
    double dt, dx, dy, omega, u_ref;
    cudaStream_t stream;
    int lanes;            // warps per 32-cell segment of the step kernel
    int prefetch;         // load path of the wall-free cells (lbm_set_variant)
    int splitting;        // LBM_SPLIT_LIE (stored state h) or LBM_SPLIT_STRANG[_EXACT] (stored g = R(dt/2) h)
    int order;            // transport order: 1 (first-order upwind, the paper's) or 2
    int grid;             // blocks of the bulk step kernel
    int march_grid;       // persistent blocks of the column-march kernel (load paths 4 to 8)
    bool tiled;           // the state buffers hold the strip-tiled layout (load paths 8, 9)
    long tile_pitch;      // floats per tile of that layout
    int nparts_step;      // residual partial slots of one step (bulk + wall kernels)
    int *wall_segs;       // device list of wall segments for the current lanes
    int wall_cap;
    // device memory
    void *base;
    bool owns;
    size_t bytes;
    void *buf[4];         // state ping-pong (0,1); refinement: defect (2), correction (3)
    int cur;              // index of the current state buffer
    double *tab64;
    float *tab32;
    TableHeader *hdr;
    double *partials;
    int npartials;
    double *result;       // [0] sum d^2, [1] sum h^2, [2] r, [3] non-finite flag
    double *moments;      // 6 * ncells
    double *flux_y;       // (ny+1) * nx
    double *flux_x;       // ny * (nx+1)
    double *host_res;     // pinned host copy of result
    StepArgs args;        // launch arguments except the buffer pointers
    cudaGraphExec_t graph[2];  // residual_every steps starting from buffer 0 / 1
    bool graph_ok[2];
    cudaStream_t cap_stream;   // private stream the graphs are captured on (created on first use)
    long step;
    long resid_step;
};

namespace {

thread_local std::string g_err;

lbm_status fail(lbm_status s, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
lbm_status fail(lbm_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

}  // namespace

// error reporting for the other translation units of the library
lbm_status lbm_norms_fail(lbm_status s, const char *msg) { return fail(s, "%s", msg); }

namespace {

lbm_status cuda_fail(cudaError_t e, const char *what)
{
    return fail(LBM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

size_t elem_size(int prec) { return prec == LBM_FP64 ? sizeof(double) : sizeof(float); }

bool kernel_m_supported(int m) { return m == 3 || m == 4 || m == 6 || m == 8 || m == 12; }

// grids the column march can take (nx a multiple of 64, at least two strips' width, ten
// rows); FP32 cavities of such grids get state buffers large enough for the strip-tiled
// layout of load paths 8 and 9 as well
bool march_grid_ok(const lbm_problem *p) { return p->nx % 64 == 0 && p->nx >= 128 && p->ny >= 10; }
bool tile_eligible(const lbm_problem *p) { return p->prec == LBM_FP32_PERTURB && p->geom == LBM_CAVITY && march_grid_ok(p); }

struct Layout {
    size_t off_buf[4];
    size_t off_tab64, off_tab32, off_hdr, off_partials, off_result, off_moments, off_fy, off_fx, off_wsegs;
    int wall_cap;
    size_t total;
    int nbuf;
    int npartials;
};

Layout make_layout(const lbm_vset *vs, const lbm_problem *p)
{
    Layout L{};
    const long ncells = (long)p->nx * p->ny;
    size_t nvals = (size_t)vs->m * vs->m * ncells;
    if (tile_eligible(p)) nvals = std::max(nvals, tiled_values(vs->m * vs->m, p->nx, p->ny));
    const size_t es = elem_size(p->prec);
    L.nbuf = (p->prec == LBM_FP64) ? 2 : 4;
    size_t off = 0;
    for (int i = 0; i < L.nbuf; ++i) {
        L.off_buf[i] = off;
        off = align256(off + nvals * es);
    }
    // FP32: buf[2] and buf[3] are adjacent, so from buf[2] on there are at least
    // 8 bytes per value: the FP64 staging area of state upload/download
    L.off_tab64 = off;
    off = align256(off + sizeof(double) * TAB_ROWS * LBM_MAX_V);
    L.off_tab32 = off;
    off = align256(off + sizeof(float) * TAB_ROWS * LBM_MAX_V);
    L.off_hdr = off;
    off = align256(off + sizeof(TableHeader));
    // segments with a wall cell: at most one per wall cell
    L.wall_cap = 2 * (p->nx + p->ny) + 4;
    L.off_wsegs = off;
    off = align256(off + sizeof(int) * L.wall_cap);
    // the finest bulk launch has one 32-cell segment per block, plus the wall kernel's
    // blocks; norms use at most 152*8 blocks
    long nb = (ncells + 31) / 32 + L.wall_cap;
    if (nb < 152 * 8) nb = 152 * 8;
    L.npartials = (int)nb;
    L.off_partials = off;
    off = align256(off + sizeof(double) * 2 * nb);
    L.off_result = off;
    off = align256(off + sizeof(double) * 16);       // result[0..3], status word at result + 8
    L.off_moments = off;
    off = align256(off + sizeof(double) * 6 * ncells);
    L.off_fy = off;
    off = align256(off + sizeof(double) * (size_t)(p->ny + 1) * p->nx);
    L.off_fx = off;
    off = align256(off + sizeof(double) * (size_t)p->ny * (p->nx + 1));
    L.total = off;
    return L;
}

lbm_status validate(const lbm_vset *vs, const lbm_problem *p)
{
    if (!vs || !p) return fail(LBM_EINVAL, "NULL velocity set or problem");
    if (p->geom != LBM_COUETTE && p->geom != LBM_CAVITY)
        return fail(LBM_EINVAL, "geom must be LBM_COUETTE or LBM_CAVITY");
    if (p->nx < 1 || p->ny < 2) return fail(LBM_EINVAL, "grid %d x %d too small", p->nx, p->ny);
    if (p->geom == LBM_CAVITY && p->nx < 2) return fail(LBM_EINVAL, "cavity needs nx >= 2");
    if ((long)p->nx * p->ny > (1L << 31)) return fail(LBM_EINVAL, "grid too large");
    if (!(p->kn > 0)) return fail(LBM_EINVAL, "Kn must be > 0 (got %g)", p->kn);
    if (!(p->cfl > 0 && p->cfl <= 1)) return fail(LBM_EINVAL, "cfl must be in (0, 1] (got %g)", p->cfl);
    if (!std::isfinite(p->u_bottom) || !std::isfinite(p->u_top))
        return fail(LBM_EINVAL, "wall speeds must be finite");
    if (p->prec != LBM_FP64 && p->prec != LBM_FP32_PERTURB)
        return fail(LBM_EINVAL, "unknown precision %d", p->prec);
    if (p->residual_every < 1) return fail(LBM_EINVAL, "residual_every must be >= 1");
    if (!kernel_m_supported(vs->m))
        return fail(LBM_EUNSUPPORTED, "no step kernel for %d nodes per axis (have 3, 4, 6, 8, 12)", vs->m);
    return LBM_OK;
}

// dt, Courant numbers, relaxation and ghost coefficients (host, FP64)
void fill_tables(lbm_sim *s, std::vector<double> &t64, std::vector<float> &t32, TableHeader &hdr)
{
    const lbm_problem &p = s->prob;
    const lbm_vset &v = s->vs;
    const int m = v.m, nv = m * m;
    double mx = 0, dxw = 0, dyw = 0;
    for (int i = 0; i < m; ++i) mx = std::fmax(mx, std::fabs(v.nodes[i]));
    for (int a = 0; a < nv; ++a) {
        if (v.xi_x[a] > 0) dxw += v.xi_x[a] * v.w[a];
        if (v.xi_y[a] > 0) dyw += v.xi_y[a] * v.w[a];
    }
    if (p.geom == LBM_COUETTE) {
        s->dy = 1.0 / p.ny;
        s->dx = s->dy;
    } else {
        s->dx = 1.0 / p.nx;
        s->dy = 1.0 / p.ny;
    }
    double rate = mx / s->dy;
    if (!(p.geom == LBM_COUETTE && p.nx == 1)) rate += mx / s->dx;
    s->dt = p.cfl / rate;
    if (std::isfinite(p.kn) && s->dt > p.kn) s->dt = p.kn;
    s->omega = std::isfinite(p.kn) ? s->dt / p.kn : 0.0;
    s->u_ref = std::fmax(std::fabs(p.u_bottom), std::fabs(p.u_top));
    if (s->u_ref == 0) s->u_ref = 1.0;

    t64.assign((size_t)TAB_ROWS * LBM_MAX_V, 0.0);
    for (int a = 0; a < nv; ++a) {
        const double nux = std::fabs(v.xi_x[a]) * s->dt / s->dx;
        const double nuy = std::fabs(v.xi_y[a]) * s->dt / s->dy;
        // a Couette column of width one cell has no x transport
        const double nux_eff = (p.geom == LBM_COUETTE && p.nx == 1) ? 0.0 : nux;
        t64[TAB_A0 * LBM_MAX_V + a] = 1.0 - nux_eff - nuy;
        t64[TAB_NUX * LBM_MAX_V + a] = nux_eff;
        t64[TAB_NUY * LBM_MAX_V + a] = nuy;
        t64[TAB_CW * LBM_MAX_V + a] = s->omega * v.w[a];
        t64[TAB_GB_LIN * LBM_MAX_V + a] = v.w[a] * (1.0 + v.xi_x[a] * p.u_bottom);
        t64[TAB_GB_C * LBM_MAX_V + a] = v.w[a] * v.xi_x[a] * p.u_bottom / s->u_ref;
        t64[TAB_GT_LIN * LBM_MAX_V + a] = v.w[a] * (1.0 + v.xi_x[a] * p.u_top);
        t64[TAB_GT_C * LBM_MAX_V + a] = v.w[a] * v.xi_x[a] * p.u_top / s->u_ref;
        t64[TAB_W * LBM_MAX_V + a] = v.w[a];
    }
    t32.resize(t64.size());
    for (size_t i = 0; i < t64.size(); ++i) t32[i] = (float)t64[i];
    std::memset(&hdr, 0, sizeof hdr);
    for (int i = 0; i < m; ++i) {
        hdr.xi1[i] = v.nodes[i];
        hdr.w1[i] = v.weights[i];
    }
    hdr.b = 1.0 - s->omega;
    hdr.inv_dx_wall = 1.0 / dxw;
    hdr.inv_dy_wall = 1.0 / dyw;
}

bool planar(const lbm_sim *s) { return s->args.pa == s->ncells; }

void drop_graphs_fwd(lbm_sim *s);

// factor of the non-equilibrium part from h to the stored g = R(dt/2) h
double half_relax_factor(const lbm_sim *s)
{
    if (s->splitting == LBM_SPLIT_STRANG_EXACT) return std::exp(-0.5 * s->omega);
    if (s->splitting == LBM_SPLIT_STRANG) return 1.0 - 0.5 * s->omega;
    return 1.0;
}

// FP64 staging area for host transfers of the state: the two spare float arrays (adjacent,
// 8 bytes per value) of an FP32 simulation, the other state buffer of an FP64 one
double *staging(lbm_sim *s, const void *state)
{
    if (s->prob.prec != LBM_FP64) return (double *)s->buf[2];
    return (double *)(state == s->buf[0] ? s->buf[1] : s->buf[0]);
}

// host FP64 [n][ny][nx] -> device state `dst` in the simulation's layout and precision
lbm_status upload_state(lbm_sim *s, const double *h, void *dst)
{
    const size_t nvals = (size_t)s->nv * s->ncells;
    cudaError_t e;
    if (s->prob.prec == LBM_FP64 && planar(s)) {
        e = cudaMemcpyAsync(dst, h, nvals * sizeof(double), cudaMemcpyHostToDevice, s->stream);
    } else {
        double *stage = staging(s, dst);
        e = cudaMemcpyAsync(stage, h, nvals * sizeof(double), cudaMemcpyHostToDevice, s->stream);
        if (e == cudaSuccess)
            e = launch_relayout(s->prob.prec, true, stage, dst, s->nv, s->prob.nx, s->prob.ny, s->args.pa,
                                s->args.py, s->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    return e == cudaSuccess ? LBM_OK : cuda_fail(e, "uploading the state");
}

// Move the current state between the planar and the strip-tiled layout (through the other
// state buffer, which the next step overwrites anyway).  Stream-ordered.
cudaError_t set_tiled(lbm_sim *s, bool tiled)
{
    if (s->tiled == tiled) return cudaSuccess;
    cudaError_t e = launch_tile_convert(tiled, (const float *)s->buf[s->cur], (float *)s->buf[s->cur ^ 1], s->nv,
                                        s->prob.nx, s->prob.ny, s->tile_pitch, s->stream);
    if (e != cudaSuccess) return e;
    s->cur ^= 1;
    s->tiled = tiled;
    s->args.tile_pitch = tiled ? s->tile_pitch : 0;
    drop_graphs_fwd(s);
    return cudaSuccess;
}

// The current state in the planar layout: the state itself, or (strip-tiled state) a planar
// copy in the other state buffer.  Stream-ordered; valid until the next step.
const void *planar_state(lbm_sim *s, cudaError_t *e)
{
    *e = cudaSuccess;
    if (!s->tiled) return s->buf[s->cur];
    *e = launch_tile_convert(false, (const float *)s->buf[s->cur], (float *)s->buf[s->cur ^ 1], s->nv, s->prob.nx,
                             s->prob.ny, s->tile_pitch, s->stream);
    return s->buf[s->cur ^ 1];
}

// Where a writer puts a planar state, and the step that makes it current: a strip-tiled
// simulation takes the planar state in the other buffer and tiles it into the current one.
void *planar_target(lbm_sim *s) { return s->tiled ? s->buf[s->cur ^ 1] : s->buf[s->cur]; }
cudaError_t commit_planar(lbm_sim *s)
{
    if (!s->tiled) return cudaSuccess;
    return launch_tile_convert(true, (const float *)s->buf[s->cur ^ 1], (float *)s->buf[s->cur], s->nv, s->prob.nx,
                               s->prob.ny, s->tile_pitch, s->stream);
}

StepArgs base_args(const lbm_sim *s) { return s->args; }

void fill_args(lbm_sim *s, const TableHeader &hdr)
{
    StepArgs &a = s->args;
    std::memset(&a, 0, sizeof a);
    const lbm_problem &p = s->prob;
    const lbm_vset &v = s->vs;
    a.partials = s->partials;
    a.status = (int *)(s->result + 8);
    a.nx = p.nx;
    a.ny = p.ny;
    a.ncells = s->ncells;
    // planar state layout [a][y][x].  A row-interleaved layout [y][a][x] (pa = nx, py = n nx),
    // which makes a row step of the interior march touch one contiguous stretch of memory,
    // measured the same march time at 2048^2 x 144, and addressing the step kernels through
    // run-time pitches cost 4-8 % of their speed, so they index the planar layout directly.
    (void)v;
    a.pa = s->ncells;
    a.py = p.nx;
    a.cavity = p.geom == LBM_CAVITY;
    a.homogeneous = 0;
    const bool column = p.geom == LBM_COUETTE && p.nx == 1;
    for (int i = 0; i < v.m; ++i) {
        a.xi[i] = v.nodes[i];
        a.nux[i] = column ? 0.0 : std::fabs(v.nodes[i]) * s->dt / s->dx;
        a.nuy[i] = std::fabs(v.nodes[i]) * s->dt / s->dy;
        a.w1[i] = v.weights[i];
        a.xi_f[i] = (float)a.xi[i];
        a.nux_f[i] = (float)a.nux[i];
        a.nuy_f[i] = (float)a.nuy[i];
        a.w1_f[i] = (float)a.w1[i];
        for (int ax = 0; ax < 2; ++ax) {
            const double nu = ax == 0 ? a.nux[i] : a.nuy[i];
            a.so_p[ax][i] = 0.5 * nu * (3.0 - nu);
            a.so_b[ax][i] = nu * (2.0 - nu);
            a.so_c[ax][i] = -0.5 * nu * (1.0 - nu);
            a.so_p_f[ax][i] = (float)a.so_p[ax][i];
            a.so_b_f[ax][i] = (float)a.so_b[ax][i];
            a.so_c_f[ax][i] = (float)a.so_c[ax][i];
        }
    }
    a.omega = s->omega;
    a.b = 1.0 - s->omega;
    a.omega_f = (float)a.omega;
    a.b_f = (float)a.b;
    a.inv_dx_wall = hdr.inv_dx_wall;
    a.inv_dy_wall = hdr.inv_dy_wall;
    a.u_bottom = p.u_bottom;
    a.u_top = p.u_top;
    a.inv_u_ref = 1.0 / s->u_ref;
}

int grid_for(long ncells, int lanes)
{
    const long cpb = 32L * segs_per_block(lanes);
    return (int)((ncells + cpb - 1) / cpb);
}

void drop_graphs(lbm_sim *s)
{
    for (int p = 0; p < 2; ++p) {
        if (s->graph_ok[p]) cudaGraphExecDestroy(s->graph[p]);
        s->graph_ok[p] = false;
    }
}

void drop_graphs_fwd(lbm_sim *s) { drop_graphs(s); }

// Enqueue steps [first, first + count) starting from buffer `cur` on `st` (no bookkeeping).
cudaError_t enqueue_steps(lbm_sim *s, long first, long count, int cur, cudaStream_t st)
{
    StepArgs a = s->args;
    for (long i = 0; i < count; ++i) {
        const long idx = first + i;
        const bool resid = idx % s->prob.residual_every == 0;
        a.h = s->buf[cur];
        a.hn = s->buf[cur ^ 1];
        cudaError_t e;
        if (s->order == 2)
            e = s->prefetch >= 8 ? launch_step_f32_so_march(s->vs.m, s->lanes, so_march_slots(s->prefetch),
                                                            so_march_tiled(s->prefetch), resid, a, s->grid, st)
                                 : launch_step_so(s->prob.prec, s->vs.m, s->lanes, resid, a, s->grid, st);
        else
            e = launch_step(s->prob.prec, s->vs.m, s->lanes, s->prefetch, resid, a, s->grid, st);
        if (e != cudaSuccess) return e;
        if (resid) {
            e = launch_finalize_residual(s->partials, s->nparts_step, s->result, st);
            if (e != cudaSuccess) return e;
        }
        cur ^= 1;
    }
    return cudaSuccess;
}

// CUDA graph of residual_every steps from buffer `cur`.  Captured on a stream private to
// the sim, never on the caller's: a caller's stream may be shared (stream pools hand the
// same stream to several users), and any work another thread enqueued on it during the
// capture would land in this graph.  The graph is launched on the caller's stream.
cudaError_t make_capture_stream(lbm_sim *s)
{
    if (s->cap_stream) return cudaSuccess;
    cudaError_t e = cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) s->cap_stream = nullptr;
    return e;
}

cudaError_t make_graph(lbm_sim *s, int cur)
{
    cudaError_t e = make_capture_stream(s);
    if (e != cudaSuccess) return e;
    cudaGraph_t g = nullptr;
    e = cudaStreamBeginCapture(s->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    const long K = s->prob.residual_every;
    cudaError_t e2 = enqueue_steps(s, 1, K, cur, s->cap_stream);   // indices 1..K: residual on the last
    e = cudaStreamEndCapture(s->cap_stream, &g);
    if (e2 != cudaSuccess || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return e2 != cudaSuccess ? e2 : e;
    }
    e = cudaGraphInstantiate(&s->graph[cur], g, 0);
    cudaGraphDestroy(g);
    if (e == cudaSuccess) s->graph_ok[cur] = true;
    return e;
}

// Select the lanes-per-cell variant: grid of the bulk kernel and the device list of
// segments (runs of 32/lanes consecutive cells, one warp each) that contain a wall cell.
lbm_status set_lanes(lbm_sim *s, int lanes)
{
    const int cpw = 32;
    const int nx = s->prob.nx, ny = s->prob.ny;
    const bool cav = s->prob.geom == LBM_CAVITY;
    std::vector<int> segs;
    auto add = [&](long c) {
        const int sg = (int)(c / cpw);
        if (segs.empty() || segs.back() != sg) segs.push_back(sg);
    };
    // wall cells in ascending order: bottom row, the side cells of each inner row (cavity),
    // top row
    // (the second-order march leaves rows 1 and ny - 2 to the wall kernel as well: their
    // face fluxes reach a wall)
    const bool rows2 = s->order == 2 && s->prefetch >= 8;
    const int whole = rows2 ? 2 : 1;   // whole rows at each end
    for (int y = 0; y < whole; ++y)
        for (int x = 0; x < nx; ++x) add((long)y * nx + x);
    for (int y = whole; y < ny - whole && cav; ++y) {
        add((long)y * nx);
        add((long)y * nx + nx - 1);
    }
    for (int y = ny - whole; y < ny; ++y)
        for (int x = 0; x < nx; ++x) add((long)y * nx + x);
    if ((int)segs.size() > s->wall_cap) return fail(LBM_EINVAL, "internal: wall segment list overflow");
    cudaError_t e = cudaMemcpyAsync(s->wall_segs, segs.data(), sizeof(int) * segs.size(),
                                    cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "uploading the wall segment list");
    drop_graphs(s);
    s->lanes = lanes;
    s->grid = grid_for(s->ncells, lanes);
    s->args.wall_segs = s->wall_segs;
    s->args.n_wall_segs = (int)segs.size();
    // one merged launch when wall segments are more than a tenth of all segments
    const long nseg_total = (s->ncells + 31) / 32;
    s->args.merged = (long)segs.size() * 10 > nseg_total ? 1 : 0;
    if (s->prefetch >= 4) {
        int strips = 0, chunks = 0;
        // every march block writes one residual partial: the march grid and the wall kernel's
        // blocks stay within the partials region (small grids of small velocity sets have
        // more resident blocks than 32-cell segments)
        const int grid = std::min(s->march_grid, s->npartials - wall_grid(lanes, (int)segs.size()));
        if (grid < 1) return fail(LBM_EINVAL, "internal: no room for the column march's residual partials");
        // the plan cuts ny - 2 interior rows; the second-order march has ny - 4
        lbm_march_plan(nx, rows2 ? ny - 2 : ny, grid, &strips, &chunks);
        s->grid = grid;
        s->args.march_strips = strips;
        s->args.march_chunks = chunks;
        s->args.counters = (int *)(s->result + 12);
        s->args.merged = 0;
    }
    s->nparts_step = s->grid + wall_grid(lanes, (int)segs.size());
    if (s->nparts_step > s->npartials) return fail(LBM_EINVAL, "internal: residual partials overflow");
    return LBM_OK;
}

}  // namespace

int default_lanes_per_cell(int prec, int m)
{
    if (prec == LBM_FP64) return m <= 4 ? 1 : (m == 6 ? 2 : 4);
    return m <= 6 ? 1 : (m == 8 ? 2 : 4);
}

// row slots of the column march's ring for load paths 4 (four), 5 (five), 6 (two slots,
// two blocks per SM) and 7 (four, relaxation deferred by one row)
// and on the strip-tiled state 8 (four slots) and 9 (four slots, bulk asynchronous stores)
static int march_slots(int pf) { return pf == 6 ? 2 : (pf == 7 || pf == 8 || pf == 9) ? 4 : pf; }
static bool march_defer(int pf) { return pf == 7; }
static int march_tiled(int pf) { return pf == 8 ? 1 : pf == 9 ? 2 : 0; }

bool step_supported(int prec, int m, int g, int pf)
{
    static const int f64[][3] = {{3, 1, 0}, {4, 1, 0}, {4, 2, 0}, {6, 1, 0}, {6, 2, 0}, {4, 2, 1}, {6, 2, 1}, {8, 2, 0}, {8, 4, 0}, {12, 3, 0}, {12, 4, 0}, {12, 6, 0}, {8, 4, 1}, {12, 6, 1}};
    static const int f32[][3] = {{3, 1, 0}, {4, 1, 0}, {6, 1, 0}, {6, 2, 0}, {8, 1, 0}, {8, 2, 0}, {8, 4, 0}, {8, 2, 1}, {8, 4, 1}, {12, 2, 0}, {12, 3, 0}, {12, 4, 0}, {12, 6, 0}, {12, 3, 1}, {12, 4, 1}, {12, 6, 1}};
    static const int tma[][2] = {{8, 2}, {8, 4}, {12, 3}, {12, 4}, {12, 6}};
    if (pf == 2 || pf == 3) {
        if (prec != LBM_FP32_PERTURB) return false;
        for (auto &v : tma) if (v[0] == m && v[1] == g) return true;
        return false;
    }
    if (pf >= 4 && pf <= 9)
        return prec == LBM_FP32_PERTURB && march_supported(m, g, march_slots(pf), march_defer(pf), march_tiled(pf));
    if (prec == LBM_FP64) {
        for (auto &v : f64) if (v[0] == m && v[1] == g && v[2] == pf) return true;
    } else {
        for (auto &v : f32) if (v[0] == m && v[1] == g && v[2] == pf) return true;
    }
    return false;
}

cudaError_t launch_step(int prec, int m, int g, int pf, bool resid, const StepArgs &a, int grid,
                        cudaStream_t s)
{
    if (pf == 2 || pf == 3) return launch_step_f32_tma(m, g, resid, a, grid, s, pf == 3);
    if (pf >= 4 && pf <= 9)
        return launch_step_f32_march(m, g, march_slots(pf), march_defer(pf), march_tiled(pf), resid, a, grid, s);
    if (prec == LBM_FP64)
        return m >= 8 ? launch_step_f64_large(m, g, pf, resid, a, grid, s)
                      : launch_step_f64_small(m, g, pf, resid, a, grid, s);
    return m >= 12 ? launch_step_f32_large(m, g, pf, resid, a, grid, s)
                   : launch_step_f32_small(m, g, pf, resid, a, grid, s);
}

extern "C" {

const char *lbm_last_error(void) { return g_err.c_str(); }

lbm_status lbm_march_plan(int nx, int ny, int blocks, int *strips, int *chunks)
{
    if (!strips || !chunks) return fail(LBM_EINVAL, "NULL argument");
    if (nx % 64 != 0 || nx < 128 || ny < 10 || blocks < 1)
        return fail(LBM_EUNSUPPORTED, "the column march needs nx a multiple of 64, nx >= 128 and ny >= 10");
    // 64-cell strips x in [32, nx - 32); the rows [1, ny - 2] cut into chunks of at least 8
    // rows (16 where the grid allows) and, where the grid allows, at least 4 items per block;
    // among those the count minimising (rounds of items x blocks) / items, the idle share of
    // the last round, times (1 + chunks / rows), the share of rows copied twice at chunk
    // boundaries
    const int S = (nx - 64) / 64, rows = ny - 2, G = blocks;
    const int lo_len = rows >= 16 * 4 ? 16 : 8;
    int cmax = rows / lo_len, cmin = (4 * G + S - 1) / S;
    if (cmax < 1) cmax = 1;
    if (cmin > cmax) cmin = cmax;
    int best_c = cmax;
    double best = 1e300;
    for (int c = cmin; c <= cmax; ++c) {
        const long items = (long)S * c;
        const long rounds = (items + G - 1) / G;
        const double cost = (double)(rounds * G) / items * (1.0 + (double)c / rows);
        if (cost < best - 1e-12) {
            best = cost;
            best_c = c;
        }
    }
    *strips = S;
    *chunks = best_c;
    return LBM_OK;
}

lbm_status lbm_stream_create(void **stream)
{
    if (!stream) return fail(LBM_EINVAL, "stream is NULL");
    cudaStream_t st = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e, "creating a stream");
    *stream = st;
    return LBM_OK;
}

void lbm_stream_destroy(void *stream)
{
    if (!stream) return;
    cudaStreamSynchronize((cudaStream_t)stream);
    cudaStreamDestroy((cudaStream_t)stream);
}

lbm_status lbm_make_velocity_set(int kind, int n, lbm_vset **out)
{
    if (!out) return fail(LBM_EINVAL, "out is NULL");
    *out = nullptr;
    if (kind != LBM_HALF_RANGE_GH && kind != LBM_FULL_RANGE_GH)
        return fail(LBM_EINVAL, "unknown velocity-set kind %d", kind);
    if (kind == LBM_HALF_RANGE_GH && (n < 1 || n > 8))
        return fail(LBM_EINVAL, "half-range sets need 1 <= N <= 8 nodes per half-axis (got %d)", n);
    if (kind == LBM_FULL_RANGE_GH && (n < 2 || n > 16))
        return fail(LBM_EINVAL, "full-range sets need 2 <= M <= 16 nodes per axis (got %d)", n);
    lbm_vset *v = new (std::nothrow) lbm_vset;
    if (!v) return fail(LBM_ENOMEM, "host allocation failed");
    v->kind = kind;
    v->n_arg = n;
    if (!lbm_rule_1d(kind, n, v->nodes, v->weights)) {
        delete v;
        return fail(LBM_EINVAL, "quadrature construction failed");
    }
    v->m = (int)v->nodes.size();
    for (int iy = 0; iy < v->m; ++iy)
        for (int ix = 0; ix < v->m; ++ix) {
            v->xi_x.push_back(v->nodes[ix]);
            v->xi_y.push_back(v->nodes[iy]);
            v->w.push_back(v->weights[ix] * v->weights[iy]);
        }
    *out = v;
    return LBM_OK;
}

lbm_status lbm_vset_query(const lbm_vset *vs, int *n_vel, int *m, double *xi_x, double *xi_y,
                          double *w)
{
    if (!vs) return fail(LBM_EINVAL, "velocity set is NULL");
    const int nv = vs->m * vs->m;
    if (n_vel) *n_vel = nv;
    if (m) *m = vs->m;
    if (xi_x) std::memcpy(xi_x, vs->xi_x.data(), sizeof(double) * nv);
    if (xi_y) std::memcpy(xi_y, vs->xi_y.data(), sizeof(double) * nv);
    if (w) std::memcpy(w, vs->w.data(), sizeof(double) * nv);
    return LBM_OK;
}

void lbm_vset_destroy(lbm_vset *vs) { delete vs; }

lbm_status lbm_sim_bytes(const lbm_vset *vs, const lbm_problem *prob, size_t *bytes)
{
    if (!bytes) return fail(LBM_EINVAL, "bytes is NULL");
    lbm_status st = validate(vs, prob);
    if (st != LBM_OK) return st;
    *bytes = make_layout(vs, prob).total;
    return LBM_OK;
}

lbm_status lbm_init(const lbm_vset *vs, const lbm_problem *prob, const double *init_h,
                    void *device_buf, size_t buf_bytes, void *stream, lbm_sim **out)
{
    if (!out) return fail(LBM_EINVAL, "out is NULL");
    *out = nullptr;
    lbm_status st = validate(vs, prob);
    if (st != LBM_OK) return st;
    Layout L = make_layout(vs, prob);
    if (device_buf) {
        if (buf_bytes < L.total)
            return fail(LBM_ENOMEM, "device buffer of %zu bytes < %zu needed", buf_bytes, L.total);
        if (((uintptr_t)device_buf) & 255) return fail(LBM_EINVAL, "device buffer must be 256-byte aligned");
    }
    lbm_sim *s = new (std::nothrow) lbm_sim;
    if (!s) return fail(LBM_ENOMEM, "host allocation failed");
    s->vs = *vs;
    s->prob = *prob;
    s->nv = vs->m * vs->m;
    s->ncells = (long)prob->nx * prob->ny;
    s->stream = (cudaStream_t)stream;
    s->lanes = default_lanes_per_cell(prob->prec, vs->m);
    s->prefetch = 0;
    s->splitting = LBM_SPLIT_LIE;
    s->order = 1;
    s->march_grid = 0;
    s->tiled = false;
    s->tile_pitch = (long)prob->ny * vs->m * vs->m * LBM_TILE_W;
    s->step = 0;
    s->resid_step = -1;
    s->cur = 0;
    s->host_res = nullptr;
    s->graph_ok[0] = s->graph_ok[1] = false;
    s->cap_stream = nullptr;
    s->owns = device_buf == nullptr;
    s->bytes = L.total;
    if (s->owns) {
        cudaError_t e = cudaMalloc(&s->base, L.total);
        if (e != cudaSuccess) {
            delete s;
            return fail(LBM_ENOMEM, "cudaMalloc of %zu bytes: %s", L.total, cudaGetErrorString(e));
        }
    } else {
        s->base = device_buf;
    }
    char *b = (char *)s->base;
    for (int i = 0; i < 4; ++i) s->buf[i] = (i < L.nbuf) ? b + L.off_buf[i] : nullptr;
    s->tab64 = (double *)(b + L.off_tab64);
    s->tab32 = (float *)(b + L.off_tab32);
    s->hdr = (TableHeader *)(b + L.off_hdr);
    s->partials = (double *)(b + L.off_partials);
    s->npartials = L.npartials;
    s->result = (double *)(b + L.off_result);
    s->moments = (double *)(b + L.off_moments);
    s->flux_y = (double *)(b + L.off_fy);
    s->flux_x = (double *)(b + L.off_fx);
    s->wall_segs = (int *)(b + L.off_wsegs);
    s->wall_cap = L.wall_cap;

    std::vector<double> t64;
    std::vector<float> t32;
    TableHeader hdr;
    fill_tables(s, t64, t32, hdr);
    fill_args(s, hdr);
    cudaError_t e = cudaMallocHost(&s->host_res, sizeof(double) * 16);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->tab64, t64.data(), sizeof(double) * t64.size(), cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->tab32, t32.data(), sizeof(float) * t32.size(), cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->hdr, &hdr, sizeof hdr, cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->result, 0, sizeof(double) * 16, s->stream);
    const size_t state_bytes = (L.off_buf[1] - L.off_buf[0]);
    if (e == cudaSuccess && !init_h) e = cudaMemsetAsync(s->buf[0], 0, state_bytes, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) {
        lbm_status r = cuda_fail(e, "initialising the simulation");
        lbm_destroy(s);
        return r;
    }
    st = set_lanes(s, s->lanes);
    if (st != LBM_OK) {
        lbm_destroy(s);
        return st;
    }
    if (init_h) {
        st = upload_state(s, init_h, s->buf[0]);
        if (st != LBM_OK) {
            lbm_destroy(s);
            return st;
        }
    }
    *out = s;
    return LBM_OK;
}

void lbm_destroy(lbm_sim *s)
{
    if (!s) return;
    if (s->stream) cudaStreamSynchronize(s->stream);
    else cudaDeviceSynchronize();
    drop_graphs(s);
    if (s->cap_stream) cudaStreamDestroy(s->cap_stream);
    if (s->owns && s->base) cudaFree(s->base);
    if (s->host_res) cudaFreeHost(s->host_res);
    delete s;
}

lbm_status lbm_coeffs(const lbm_sim *s, double *dt, double *omega, double *u_ref)
{
    if (!s) return fail(LBM_EINVAL, "sim is NULL");
    if (dt) *dt = s->dt;
    if (omega) *omega = s->omega;
    if (u_ref) *u_ref = s->u_ref;
    return LBM_OK;
}

lbm_status lbm_step(lbm_sim *s, long nsteps)
{
    if (!s) return fail(LBM_EINVAL, "sim is NULL");
    if (nsteps < 0) return fail(LBM_EINVAL, "nsteps must be >= 0");
    const long K = s->prob.residual_every;
    // whole residual intervals replay a captured graph (not on the legacy stream, and not
    // while the caller is capturing this stream: then the launches go into their graph)
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    bool graphs = s->stream != nullptr && K >= 2;
    if (graphs && cudaStreamIsCapturing(s->stream, &cap) != cudaSuccess) graphs = false;
    if (cap != cudaStreamCaptureStatusNone) graphs = false;
    long i = 0;
    while (i < nsteps) {
        if (graphs && s->step % K == 0 && nsteps - i >= K) {
            const int p = s->cur;
            if (!s->graph_ok[p]) {
                cudaError_t e = make_graph(s, p);
                if (e != cudaSuccess) {
                    cudaGetLastError();
                    graphs = false;
                    continue;
                }
            }
            cudaError_t e = cudaGraphLaunch(s->graph[p], s->stream);
            if (e != cudaSuccess) return cuda_fail(e, "launching the step graph");
            s->cur = p ^ (int)(K & 1);
            s->step += K;
            s->resid_step = s->step;
            i += K;
            continue;
        }
        const long idx = s->step + 1;
        cudaError_t e = enqueue_steps(s, idx, 1, s->cur, s->stream);
        if (e != cudaSuccess) return cuda_fail(e, "launching the step kernels");
        if (idx % K == 0) s->resid_step = idx;
        s->cur ^= 1;
        s->step = idx;
        ++i;
    }
    return LBM_OK;
}

namespace {

lbm_status read_result(lbm_sim *s, double out[4])
{
    cudaError_t e = cudaMemcpyAsync(s->host_res, s->result, sizeof(double) * 4,
                                    cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "reading a reduction result");
    for (int k = 0; k < 4; ++k) out[k] = s->host_res[k];
    if (out[3] != 0.0) return fail(LBM_ENONFINITE, "non-finite values met in a reduction");
    return LBM_OK;
}

int nparts_for(const lbm_sim *s, int lanes)
{
    return grid_for(s->ncells, lanes) + wall_grid(lanes, s->args.n_wall_segs);
}

// FP64 defect of the FP32 state H: D = M64(H) - H (float); returns ||D||^2, ||M64(H)||^2.
lbm_status defect_pass(lbm_sim *s, void *H, void *D, double *dsum, double *nsum)
{
    StepArgs a = s->args;
    a.h = H;
    a.hn = D;
    const int g = defect_lanes(s->vs.m);
    cudaError_t e = launch_defect_f32(s->vs.m, a, grid_for(s->ncells, g), s->stream);
    if (e == cudaSuccess) e = launch_finalize_residual(s->partials, nparts_for(s, g), s->result, s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "launching the defect pass");
    double r[4];
    lbm_status st = read_result(s, r);
    if (st != LBM_OK) return st;
    *dsum = r[0];
    *nsum = r[1];
    return LBM_OK;
}

}  // namespace

lbm_status lbm_solve(lbm_sim *s, double tol, long max_steps, int refine_sweeps, double refine_tol,
                     lbm_solve_info *info)
{
    if (!s) return fail(LBM_EINVAL, "sim is NULL");
    if (!(tol > 0) || max_steps < 0 || refine_sweeps < 0) return fail(LBM_EINVAL, "invalid solve arguments");
    if (refine_sweeps > 0 && s->prob.prec != LBM_FP32_PERTURB)
        return fail(LBM_EINVAL, "refinement sweeps apply to the FP32 precision only");
    if (refine_sweeps > 0 && s->order == 2)
        return fail(LBM_EUNSUPPORTED, "the refinement kernels implement the first-order transport only");
    lbm_solve_info out{};
    const long K = s->prob.residual_every;
    // --- the march: whole residual intervals until r < tol ---
    // An FP32 march cannot push its per-step change below its rounding floor (~1e-8 of
    // ||h|| on a 128^2 cavity): with refinement it stops at max(tol, 5e-8) -- as deep as the
    // FP32 march goes without stalling, since its steps are cheaper than the correction's --
    // and leaves the rest to the FP64 defect correction; in any precision it stops when the
    // residual has not improved by 1 % over 20 consecutive checks (stagnation at the floor).
    const bool fp32_refined = refine_sweeps > 0;
    const double tol_march = fp32_refined ? std::fmax(tol, 5e-8) : tol;
    double r = INFINITY, best = INFINITY;
    int flat = 0;
    long taken = 0;
    while (taken < max_steps) {
        const long todo = K - (s->step % K);
        lbm_status st = lbm_step(s, todo);
        if (st != LBM_OK) return st;
        taken += todo;
        long rs;
        st = lbm_residual(s, &r, &rs);
        if (st != LBM_OK) return st;
        if (r < tol_march) break;
        if (r < 0.99 * best) {
            best = r;
            flat = 0;
        } else if (++flat >= 20) {
            break;
        }
    }
    out.steps = taken;
    out.residual = r;
    out.defect = r;
    // --- FP32: mixed-precision refinement (defect in FP64, correction march in FP32) ---
    // (on the planar state: a strip-tiled one is moved back to that layout afterwards)
    const bool was_tiled = s->tiled;
    if (refine_sweeps > 0 && was_tiled) {
        cudaError_t e = set_tiled(s, false);
        if (e != cudaSuccess) return cuda_fail(e, "moving the state to the planar layout");
    }
    if (refine_sweeps > 0) {
        void *H = s->buf[s->cur];
        void *D = s->buf[2];
        double dsum, nsum;
        lbm_status st = defect_pass(s, H, D, &dsum, &nsum);
        if (st != LBM_OK) return st;
        double r64 = nsum > 0 ? std::sqrt(dsum / nsum) : 0.0;
        const double hnorm = std::sqrt(nsum);
        const int g = correct_lanes(s->vs.m);
        const int grid = grid_for(s->ncells, g), nparts = nparts_for(s, g);
        const double ctol = refine_tol > 0 ? refine_tol : 0.1 * tol;
        const size_t state_bytes = (size_t)s->nv * s->ncells * sizeof(float);
        // sweeps until the FP64 defect -- the FP64 march's own residual, evaluated on the
        // refined state -- is below tol
        for (int sw = 0; sw < refine_sweeps && r64 >= tol && hnorm > 0; ++sw) {
            // correction march delta <- L(delta) + D from delta = 0 (homogeneous walls)
            void *C[2] = {s->buf[s->cur ^ 1], s->buf[3]};
            int cc = 0;
            cudaError_t e = cudaMemsetAsync(C[0], 0, state_bytes, s->stream);
            if (e != cudaSuccess) return cuda_fail(e, "clearing the correction");
            StepArgs a = s->args;
            a.src = D;
            a.homogeneous = 1;
            // one interval of K correction steps (+ the residual finalisation) from C[p]
            auto enqueue_interval = [&](int p, cudaStream_t st) -> cudaError_t {
                int q = p;
                for (long j = 1; j <= K; ++j) {
                    StepArgs b = a;
                    b.h = C[q];
                    b.hn = C[q ^ 1];
                    cudaError_t err = launch_correct_f32(s->vs.m, g, j == K, b, grid, st);
                    if (err == cudaSuccess && j == K)
                        err = launch_finalize_residual(s->partials, nparts, s->result, st);
                    if (err != cudaSuccess) return err;
                    q ^= 1;
                }
                return cudaSuccess;
            };
            // the intervals replay CUDA graphs (captured on the private stream, one per
            // starting buffer); direct launches if a capture fails
            cudaGraphExec_t cg[2] = {nullptr, nullptr};
            bool use_graphs = K >= 2 && make_capture_stream(s) == cudaSuccess;
            long k = 0;
            double cbest = INFINITY;
            int cflat = 0;
            while (k < max_steps) {
                if (use_graphs && !cg[cc]) {
                    cudaGraph_t gr = nullptr;
                    cudaError_t ec = cudaStreamBeginCapture(s->cap_stream, cudaStreamCaptureModeThreadLocal);
                    if (ec == cudaSuccess) {
                        cudaError_t e2 = enqueue_interval(cc, s->cap_stream);
                        ec = cudaStreamEndCapture(s->cap_stream, &gr);
                        if (e2 != cudaSuccess) ec = e2;
                    }
                    if (ec == cudaSuccess) ec = cudaGraphInstantiate(&cg[cc], gr, 0);
                    if (gr) cudaGraphDestroy(gr);
                    if (ec != cudaSuccess) {
                        cudaGetLastError();
                        cg[cc] = nullptr;
                        use_graphs = false;
                    }
                }
                e = use_graphs ? cudaGraphLaunch(cg[cc], s->stream) : enqueue_interval(cc, s->stream);
                if (e != cudaSuccess) {
                    for (auto &x : cg)
                        if (x) cudaGraphExecDestroy(x);
                    return cuda_fail(e, "launching the correction march");
                }
                cc ^= (int)(K & 1);
                k += K;
                double rr[4];
                st = read_result(s, rr);
                if (st != LBM_OK) {
                    for (auto &x : cg)
                        if (x) cudaGraphExecDestroy(x);
                    return st;
                }
                // change per step relative to ||h||, 10x below tol: the correction's own error
                // is its per-step change times the conditioning of the slow modes (~1e3)
                const double change = std::sqrt(rr[0]) / hnorm;
                if (change < ctol) break;
                if (change < 0.99 * cbest) {
                    cbest = change;
                    cflat = 0;
                } else if (++cflat >= 20) {
                    break;
                }
            }
            for (auto &x : cg)
                if (x) cudaGraphExecDestroy(x);
            out.correction_steps += k;
            e = launch_add_f32((float *)H, (const float *)C[cc], (long)s->nv * s->ncells, s->stream);
            if (e != cudaSuccess) return cuda_fail(e, "applying the correction");
            out.sweeps = sw + 1;
            const double prev = r64;
            st = defect_pass(s, H, D, &dsum, &nsum);
            if (st != LBM_OK) return st;
            r64 = nsum > 0 ? std::sqrt(dsum / nsum) : 0.0;
            if (r64 > 0.5 * prev) break;      // at the FP32 rounding floor
        }
        out.defect = r64;
    }
    if (refine_sweeps > 0 && was_tiled) {
        cudaError_t e = set_tiled(s, true);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
        if (e != cudaSuccess) return cuda_fail(e, "moving the state to the strip-tiled layout");
    }
    if (info) *info = out;
    return LBM_OK;
}

lbm_status lbm_warm_start(lbm_sim *s, lbm_mlp *mlp, double kn, double u_w)
{
    if (!s || !mlp) return fail(LBM_EINVAL, "NULL argument");
    if (s->prob.geom != LBM_CAVITY) return fail(LBM_EINVAL, "the warm-start network is trained on cavities");
    float *feat = (float *)s->moments;                  // scratch: 16 B + 24 B per cell <= 48 B
    float *pred = feat + 4 * s->ncells;
    // the network runs on its own stream: its inputs/outputs live in this sim's scratch
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "warm start");
    lbm_status st = lbm_mlp_features(mlp, s->prob.nx, s->prob.ny, kn, u_w, feat);
    if (st == LBM_OK) st = lbm_mlp_forward(mlp, feat, (int)s->ncells, pred);
    if (st != LBM_OK) return st;
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "warm start");
    e = launch_warm_state(pred, s->prob.nx, s->prob.ny, s->args.pa, s->args.py, s->vs.m, s->hdr->xi1, s->hdr->w1,
                          u_w / s->u_ref, planar_target(s), s->prob.prec, s->stream);
    if (e == cudaSuccess) e = commit_planar(s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    return e == cudaSuccess ? LBM_OK : cuda_fail(e, "building the warm-start state");
}

// Second-order transport: the segment kernel of step_so.cuh (load path 0, its fixed warps
// per segment), or on FP32 cavities the second-order column march on the strip-tiled state
// (load paths 8 and 9).
static lbm_status set_variant_order2(lbm_sim *s, int warps_per_segment, int prefetch)
{
    const int m = s->vs.m;
    if (prefetch == 0) {
        if (!so_supported(s->prob.prec, m, warps_per_segment))
            return fail(LBM_EUNSUPPORTED, "no second-order segment kernel with %d warps per segment for M = %d",
                        warps_per_segment, m);
    } else if (prefetch == 8 || prefetch == 9) {
        if (!so_march_supported(m, warps_per_segment, so_march_slots(prefetch), so_march_tiled(prefetch)))
            return fail(LBM_EUNSUPPORTED, "no second-order column march with %d warps per segment (load path %d) for M = %d",
                        warps_per_segment, prefetch, m);
        if (!tile_eligible(&s->prob) || s->prob.ny < 12)
            return fail(LBM_EUNSUPPORTED, "the second-order column march needs an FP32 cavity with nx a multiple of 64, "
                                          "nx >= 128 and ny >= 12");
        int grid = 0;
        cudaError_t e = prepare_step_f32_so_march(m, warps_per_segment, so_march_slots(prefetch),
                                                  so_march_tiled(prefetch), &grid);
        if (e != cudaSuccess) return cuda_fail(e, "enabling the second-order column march's shared memory");
        if (grid <= 0) return fail(LBM_EUNSUPPORTED, "the second-order column march does not fit on an SM");
        s->march_grid = grid;
    } else {
        return fail(LBM_EUNSUPPORTED, "the second-order transport has load paths 0, 8 and 9");
    }
    cudaError_t e = set_tiled(s, prefetch != 0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "changing the state layout");
    s->prefetch = prefetch;
    return set_lanes(s, warps_per_segment);
}

lbm_status lbm_set_variant(lbm_sim *s, int warps_per_segment, int prefetch)
{
    if (!s) return fail(LBM_EINVAL, "sim is NULL");
    if (prefetch < 0 || prefetch > 9) return fail(LBM_EINVAL, "load path must be 0 to 9");
    if (s->order == 2) return set_variant_order2(s, warps_per_segment, prefetch);
    if (!step_supported(s->prob.prec, s->vs.m, warps_per_segment, prefetch))
        return fail(LBM_EUNSUPPORTED, "no step kernel with %d warps per segment (prefetch %d) for M = %d",
                    warps_per_segment, prefetch, s->vs.m);
    if (prefetch >= 2 && (s->prob.geom != LBM_CAVITY || s->prob.nx % 4 != 0 || s->ncells % 4 != 0))
        return fail(LBM_EUNSUPPORTED, "TMA staging needs a cavity with nx and the cell count multiples of 4");
    if ((prefetch == 2 || prefetch == 3) && !planar(s))
        return fail(LBM_EUNSUPPORTED, "the TMA segment kernels need the planar state layout (nx < 64)");
    if (prefetch >= 4 && !march_grid_ok(&s->prob))
        return fail(LBM_EUNSUPPORTED, "the column march needs nx a multiple of 64, nx >= 128 and ny >= 10");
    if (march_tiled(prefetch) != 0 && !tile_eligible(&s->prob))
        return fail(LBM_EUNSUPPORTED, "the strip-tiled march needs an FP32 cavity");
    if (prefetch == 2 || prefetch == 3) {
        cudaError_t e = prepare_step_f32_tma(s->vs.m, warps_per_segment);
        if (e != cudaSuccess) return cuda_fail(e, "enabling the TMA kernel's shared memory");
    }
    if (prefetch >= 4) {
        int grid = 0;
        cudaError_t e = prepare_step_f32_march(s->vs.m, warps_per_segment, march_slots(prefetch), march_defer(prefetch),
                                               march_tiled(prefetch), &grid);
        if (e != cudaSuccess) return cuda_fail(e, "enabling the column-march kernel's shared memory");
        if (grid <= 0) return fail(LBM_EUNSUPPORTED, "the column-march kernel does not fit on an SM");
        s->march_grid = grid;
    }
    // load paths 8 and 9 march the strip-tiled state, every other path the planar one
    cudaError_t e = set_tiled(s, march_tiled(prefetch) != 0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "changing the state layout");
    s->prefetch = prefetch;
    return set_lanes(s, warps_per_segment);
}

lbm_status lbm_set_splitting(lbm_sim *s, int scheme)
{
    if (!s) return fail(LBM_EINVAL, "sim is NULL");
    if (scheme != LBM_SPLIT_LIE && scheme != LBM_SPLIT_STRANG && scheme != LBM_SPLIT_STRANG_EXACT)
        return fail(LBM_EINVAL, "splitting must be LBM_SPLIT_LIE, LBM_SPLIT_STRANG or LBM_SPLIT_STRANG_EXACT");
    if (s->step != 0) return fail(LBM_EINVAL, "the splitting is chosen before the first step");
    s->splitting = scheme;
    // relaxation factor of the stored state per step: Lie h' = (1 - w) h* + w E(h*);
    // Strang, stored g = R(dt/2) h, two half relaxations around each transport:
    // g' = (1 - w/2)^2 g* + (1 - (1 - w/2)^2) E(g*), relaxation conserving rho' and j'
    // exact half relaxations: g' = E + exp(-omega) (g* - E)
    const double w = s->omega;
    const double b = scheme == LBM_SPLIT_STRANG ? (1.0 - 0.5 * w) * (1.0 - 0.5 * w)
                   : scheme == LBM_SPLIT_STRANG_EXACT ? std::exp(-w) : 1.0 - w;
    s->args.b = b;
    s->args.omega = 1.0 - b;
    s->args.b_f = (float)b;
    s->args.omega_f = (float)(1.0 - b);
    drop_graphs(s);
    return LBM_OK;
}

lbm_status lbm_set_transport(lbm_sim *s, int order)
{
    if (!s) return fail(LBM_EINVAL, "sim is NULL");
    if (order != 1 && order != 2) return fail(LBM_EINVAL, "transport order must be 1 or 2");
    if (s->step != 0) return fail(LBM_EINVAL, "the transport order is chosen before the first step");
    s->order = order;
    s->prefetch = 0;
    cudaError_t e = set_tiled(s, false);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "changing the state layout");
    // warps per segment of the second-order segment kernel: six for D2Q^h_144 (two velocity
    // rows a warp; four left one block of eight warps per SM at 176 registers in FP64)
    const int lanes = order == 2 && s->vs.m == 12 ? 6 : default_lanes_per_cell(s->prob.prec, s->vs.m);
    return set_lanes(s, lanes);
}

lbm_status lbm_get_transport(const lbm_sim *s, int *order)
{
    if (!s || !order) return fail(LBM_EINVAL, "NULL argument");
    *order = s->order;
    return LBM_OK;
}

lbm_status lbm_get_splitting(const lbm_sim *s, int *scheme)
{
    if (!s || !scheme) return fail(LBM_EINVAL, "NULL argument");
    *scheme = s->splitting;
    return LBM_OK;
}

lbm_status lbm_get_variant(const lbm_sim *s, int *warps_per_segment, int *prefetch)
{
    if (!s) return fail(LBM_EINVAL, "NULL argument");
    if (warps_per_segment) *warps_per_segment = s->lanes;
    if (prefetch) *prefetch = s->prefetch;
    return LBM_OK;
}

lbm_status lbm_residual(lbm_sim *s, double *r, long *step)
{
    if (!s) return fail(LBM_EINVAL, "sim is NULL");
    cudaError_t e = cudaMemcpyAsync(s->host_res, s->result, sizeof(double) * 9,
                                    cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "reading the residual");
    int status;
    std::memcpy(&status, s->host_res + 8, sizeof status);
    if (status != 0) return fail(LBM_ETIMEOUT, "a device-side wait of the step kernel gave up");
    if (r) *r = s->resid_step < 0 ? INFINITY : s->host_res[2];
    if (step) *step = s->resid_step;
    if (s->resid_step >= 0 && s->host_res[3] != 0.0)
        return fail(LBM_ENONFINITE, "non-finite values in the state at step %ld", s->resid_step);
    return LBM_OK;
}

lbm_status lbm_moments(lbm_sim *s, double *rho, double *ux, double *uy, double *pxx,
                       double *pxy, double *pyy, double *wall_shear)
{
    if (!s) return fail(LBM_EINVAL, "sim is NULL");
    const int m = s->vs.m;
    cudaError_t e = cudaSuccess;
    const bool want_p = pxx || pxy || pyy;
    // the moments read a strip-tiled state in place; the wall fluxes take the planar copy
    const void *hs = nullptr;
    if (wall_shear || !s->tiled) hs = planar_state(s, &e);
    if (e == cudaSuccess) {
        if (s->tiled)
            e = launch_moments(s->prob.prec, s->buf[s->cur], s->args.pa, s->args.py, s->tab64, s->hdr, m, s->prob.nx,
                               s->prob.ny, s->u_ref, s->moments, s->stream, s->tile_pitch, want_p);
        else
            e = launch_moments(s->prob.prec, hs, s->args.pa, s->args.py, s->tab64, s->hdr, m, s->prob.nx, s->prob.ny,
                               s->u_ref, s->moments, s->stream, 0, want_p);
    }
    if (e != cudaSuccess) return cuda_fail(e, "launching the moments kernel");
    double *outs[6] = {rho, ux, uy, pxx, pxy, pyy};
    std::vector<double> tmp;
    const bool strang = s->splitting != LBM_SPLIT_LIE;
    if (strang && (pxx || pxy || pyy)) {
        // physical P from the stored half-relaxed state: non-equilibrium part / (1 - omega/2)
        tmp.resize((size_t)6 * s->ncells);
        e = cudaMemcpyAsync(tmp.data(), s->moments, sizeof(double) * tmp.size(), cudaMemcpyDeviceToHost, s->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
        if (e != cudaSuccess) return cuda_fail(e, "copying moments");
        const long n = s->ncells;
        const double f = 1.0 / half_relax_factor(s);
        for (long c = 0; c < n; ++c) {
            const double r = tmp[c];
            tmp[3 * n + c] = r + f * (tmp[3 * n + c] - r);
            tmp[4 * n + c] = f * tmp[4 * n + c];
            tmp[5 * n + c] = r + f * (tmp[5 * n + c] - r);
        }
        for (int k = 0; k < 6; ++k)
            if (outs[k]) std::memcpy(outs[k], tmp.data() + (size_t)k * n, sizeof(double) * n);
    } else {
        for (int k = 0; k < 6; ++k) {
            if (!outs[k]) continue;
            e = cudaMemcpyAsync(outs[k], s->moments + (size_t)k * s->ncells, sizeof(double) * s->ncells,
                                cudaMemcpyDeviceToHost, s->stream);
            if (e != cudaSuccess) return cuda_fail(e, "copying moments");
        }
    }
    if (wall_shear) {
        const int nx = s->prob.nx, ny = s->prob.ny;
        const bool cav = s->prob.geom == LBM_CAVITY;
        e = s->order == 2
            ? launch_face_flux2(s->prob.prec, hs, s->args.pa, s->args.py, s->tab64, s->hdr, m, nx, ny,
                                cav, s->u_ref, s->flux_y, s->flux_x, s->stream)
            : launch_face_flux(s->prob.prec, hs, s->args.pa, s->args.py, s->tab64, s->hdr, m, nx, ny,
                               cav, s->u_ref, s->flux_y, s->flux_x, nullptr, s->stream);
        if (e != cudaSuccess) return cuda_fail(e, "launching the face-flux kernel");
        std::vector<double> fy((size_t)(ny + 1) * nx), fx(cav ? (size_t)ny * (nx + 1) : 0);
        e = cudaMemcpyAsync(fy.data(), s->flux_y, sizeof(double) * fy.size(), cudaMemcpyDeviceToHost, s->stream);
        if (e == cudaSuccess && cav)
            e = cudaMemcpyAsync(fx.data(), s->flux_x, sizeof(double) * fx.size(), cudaMemcpyDeviceToHost, s->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
        if (e != cudaSuccess) return cuda_fail(e, "copying face fluxes");
        double sb = 0, st = 0, sl = 0, sr = 0;
        for (int x = 0; x < nx; ++x) {
            sb += fy[x];
            st += fy[(size_t)ny * nx + x];
        }
        if (cav)
            for (int y = 0; y < ny; ++y) {
                sl += fx[(size_t)y * (nx + 1)];
                sr += fx[(size_t)y * (nx + 1) + nx];
            }
        wall_shear[0] = sb / nx;
        wall_shear[1] = st / nx;
        wall_shear[2] = cav ? sl / ny : 0.0;
        wall_shear[3] = cav ? sr / ny : 0.0;
    }
    e = cudaStreamSynchronize(s->stream);
    return e == cudaSuccess ? LBM_OK : cuda_fail(e, "moments");
}

lbm_status lbm_face_flux(lbm_sim *s, double *flux_y, double *flux_x)
{
    if (!s) return fail(LBM_EINVAL, "sim is NULL");
    const int nx = s->prob.nx, ny = s->prob.ny;
    const bool cav = s->prob.geom == LBM_CAVITY;
    if (flux_x && !cav) return fail(LBM_EINVAL, "flux_x is defined for the cavity only");
    cudaError_t e;
    const void *hs = planar_state(s, &e);
    if (e == cudaSuccess)
        e = s->order == 2
            ? launch_face_flux2(s->prob.prec, hs, s->args.pa, s->args.py, s->tab64, s->hdr, s->vs.m, nx, ny,
                                cav, s->u_ref, s->flux_y, s->flux_x, s->stream)
            : launch_face_flux(s->prob.prec, hs, s->args.pa, s->args.py, s->tab64, s->hdr,
                               s->vs.m, nx, ny, cav, s->u_ref, s->flux_y, s->flux_x, nullptr, s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "launching the face-flux kernel");
    if (flux_y)
        e = cudaMemcpyAsync(flux_y, s->flux_y, sizeof(double) * (size_t)(ny + 1) * nx,
                            cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess && flux_x)
        e = cudaMemcpyAsync(flux_x, s->flux_x, sizeof(double) * (size_t)ny * (nx + 1),
                            cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    return e == cudaSuccess ? LBM_OK : cuda_fail(e, "face fluxes");
}

lbm_status lbm_get_state(lbm_sim *s, double *h)
{
    if (!s || !h) return fail(LBM_EINVAL, "NULL argument");
    const size_t nvals = (size_t)s->nv * s->ncells;
    cudaError_t e;
    if (s->prob.prec == LBM_FP64 && planar(s)) {
        e = cudaMemcpyAsync(h, s->buf[s->cur], nvals * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
    } else {
        // the staging area of an FP64 simulation is its other state buffer, which the next
        // step overwrites anyway
        double *stage = staging(s, s->buf[s->cur]);
        const void *hs = planar_state(s, &e);
        if (e == cudaSuccess)
            e = launch_relayout(s->prob.prec, false, stage, const_cast<void *>(hs), s->nv, s->prob.nx, s->prob.ny,
                                s->args.pa, s->args.py, s->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h, stage, nvals * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    return e == cudaSuccess ? LBM_OK : cuda_fail(e, "reading the state");
}

lbm_status lbm_set_state(lbm_sim *s, const double *h)
{
    if (!s || !h) return fail(LBM_EINVAL, "NULL argument");
    lbm_status st = upload_state(s, h, planar_target(s));
    if (st != LBM_OK || !s->tiled) return st;
    cudaError_t e = commit_planar(s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    return e == cudaSuccess ? LBM_OK : cuda_fail(e, "tiling the state");
}

// Host FP32 planar state -> the strip-tiled current state, through the planar copy in the
// other buffer, in chunks of velocity planes: the copies run on the sim's private stream and
// each chunk is tiled on the sim's stream as soon as it has landed, so that the tiling
// overlaps the next chunk's copy (the host link, not the tiling, then sets the time).
// Stream-ordered after the work already on the sim's stream.
cudaError_t upload_tiled_f32(lbm_sim *s, const float *h, float *planar)
{
    constexpr int NCHUNK = 8;
    cudaError_t e = make_capture_stream(s);
    if (e != cudaSuccess) return e;
    cudaEvent_t ev[NCHUNK + 1];
    int made = 0;
    for (; made <= NCHUNK && e == cudaSuccess; ++made) e = cudaEventCreateWithFlags(&ev[made], cudaEventDisableTiming);
    if (e != cudaSuccess) --made;
    if (e == cudaSuccess) e = cudaEventRecord(ev[NCHUNK], s->stream);         // earlier work on the sim's stream
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s->cap_stream, ev[NCHUNK], 0);
    const int n = s->nv;
    for (int k = 0; k < NCHUNK && e == cudaSuccess; ++k) {
        const int a0 = (int)((long)n * k / NCHUNK), a1 = (int)((long)n * (k + 1) / NCHUNK);
        if (a1 == a0) continue;
        const size_t off = (size_t)a0 * s->ncells, cnt = (size_t)(a1 - a0) * s->ncells;
        e = cudaMemcpyAsync(planar + off, h + off, cnt * sizeof(float), cudaMemcpyHostToDevice, s->cap_stream);
        if (e == cudaSuccess) e = cudaEventRecord(ev[k], s->cap_stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s->stream, ev[k], 0);
        if (e == cudaSuccess)
            e = launch_tile_convert_range(true, planar, (float *)s->buf[s->cur], n, a0, a1 - a0, s->prob.nx,
                                          s->prob.ny, s->tile_pitch, s->stream);
    }
    // a copy still in flight after an error must not outlive the call (the host buffer is
    // the caller's); events may be destroyed with work pending on them (release is deferred)
    if (e != cudaSuccess) cudaStreamSynchronize(s->cap_stream);
    for (int k = 0; k < made; ++k) cudaEventDestroy(ev[k]);
    return e;
}

// FP32 host transfers: an FP32 simulation's stored values move as they are (half the bytes
// of the FP64 transfers); an FP64 simulation rounds on the way out and widens on the way in,
// through its other state buffer (FP64 states are never tiled)
lbm_status lbm_get_state_f32(lbm_sim *s, float *h)
{
    if (!s || !h) return fail(LBM_EINVAL, "NULL argument");
    const size_t nvals = (size_t)s->nv * s->ncells;
    cudaError_t e = cudaSuccess;
    if (s->prob.prec == LBM_FP64) {
        float *stage = reinterpret_cast<float *>(staging(s, s->buf[s->cur]));
        e = launch_convert((const double *)s->buf[s->cur], stage, (long)nvals, s->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h, stage, nvals * sizeof(float), cudaMemcpyDeviceToHost, s->stream);
    } else {
        const void *hs = planar_state(s, &e);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h, hs, nvals * sizeof(float), cudaMemcpyDeviceToHost, s->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    return e == cudaSuccess ? LBM_OK : cuda_fail(e, "reading the state");
}

lbm_status lbm_set_state_f32(lbm_sim *s, const float *h)
{
    if (!s || !h) return fail(LBM_EINVAL, "NULL argument");
    const size_t nvals = (size_t)s->nv * s->ncells;
    void *dst = planar_target(s);
    cudaError_t e;
    if (s->prob.prec == LBM_FP64) {
        float *stage = reinterpret_cast<float *>(staging(s, dst));
        e = cudaMemcpyAsync(stage, h, nvals * sizeof(float), cudaMemcpyHostToDevice, s->stream);
        if (e == cudaSuccess) e = launch_widen(stage, (double *)dst, (long)nvals, s->stream);
    } else if (!s->tiled) {
        e = cudaMemcpyAsync(dst, h, nvals * sizeof(float), cudaMemcpyHostToDevice, s->stream);
    } else {
        e = upload_tiled_f32(s, h, (float *)dst);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    return e == cudaSuccess ? LBM_OK : cuda_fail(e, "uploading the state");
}

lbm_status lbm_set_moments(lbm_sim *s, const double *moments)
{
    if (!s || !moments) return fail(LBM_EINVAL, "NULL argument");
    std::vector<double> conv;
    if (s->splitting != LBM_SPLIT_LIE) {
        // the stored state is the half-relaxed one: its non-equilibrium part of P is
        // (1 - omega/2) (Euler) or exp(-omega/2) (exact) times the physical one (rho and j
        // are not changed by relaxation)
        const long n = s->ncells;
        const double f = half_relax_factor(s);
        conv.assign(moments, moments + 6 * n);
        for (long c = 0; c < n; ++c) {
            const double rho = conv[c];
            conv[3 * n + c] = rho + f * (conv[3 * n + c] - rho);
            conv[4 * n + c] = f * conv[4 * n + c];
            conv[5 * n + c] = rho + f * (conv[5 * n + c] - rho);
        }
        moments = conv.data();
    }
    cudaError_t e = cudaMemcpyAsync(s->moments, moments, sizeof(double) * 6 * s->ncells, cudaMemcpyHostToDevice,
                                    s->stream);
    if (e == cudaSuccess)
        e = launch_moments_state(s->prob.prec, s->moments, s->prob.nx, s->prob.ny, s->args.pa, s->args.py, s->vs.m,
                                 s->hdr, s->u_ref, planar_target(s), s->stream);
    if (e == cudaSuccess) e = commit_planar(s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    return e == cudaSuccess ? LBM_OK : cuda_fail(e, "building the state from moments");
}

lbm_status lbm_state_device(lbm_sim *s, void **ptr, long *step)
{
    if (!s) return fail(LBM_EINVAL, "sim is NULL");
    if (ptr) *ptr = s->buf[s->cur];
    if (step) *step = s->step;
    return LBM_OK;
}

lbm_status lbm_state_layout(const lbm_sim *s, long *plane_pitch, long *row_pitch)
{
    if (!s) return fail(LBM_EINVAL, "sim is NULL");
    if (s->tiled)
        return fail(LBM_EUNSUPPORTED, "the state is strip-tiled (load path 8 or 9): see lbm_state_tiling");
    if (plane_pitch) *plane_pitch = s->args.pa;
    if (row_pitch) *row_pitch = s->args.py;
    return LBM_OK;
}

lbm_status lbm_state_tiling(const lbm_sim *s, int *tile_width, int *x_shift, long *tile_pitch, long *row_pitch)
{
    if (!s) return fail(LBM_EINVAL, "sim is NULL");
    if (tile_width) *tile_width = s->tiled ? LBM_TILE_W : 0;
    if (x_shift) *x_shift = s->tiled ? LBM_TILE_SHIFT : 0;
    if (tile_pitch) *tile_pitch = s->tiled ? s->tile_pitch : 0;
    if (row_pitch) *row_pitch = s->tiled ? (long)s->nv * LBM_TILE_W : 0;
    return LBM_OK;
}

lbm_status lbm_norms_scratch_bytes(long count, size_t *bytes)
{
    if (!bytes || count < 0) return fail(LBM_EINVAL, "invalid argument");
    *bytes = sizeof(double) * 2 * (size_t)norms_blocks(count);
    return LBM_OK;
}

lbm_status lbm_norms(const void *a, const void *b, long count, int prec, void *scratch,
                     size_t scratch_bytes, double *out, void *stream)
{
    if (!a || !scratch || !out) return fail(LBM_EINVAL, "NULL argument");
    if (count < 0) return fail(LBM_EINVAL, "count must be >= 0");
    if (prec != LBM_FP64 && prec != LBM_FP32_PERTURB) return fail(LBM_EINVAL, "unknown precision %d", prec);
    const int nb = norms_blocks(count);
    if (scratch_bytes < sizeof(double) * 2 * (size_t)nb)
        return fail(LBM_ENOMEM, "scratch of %zu bytes < %zu needed", scratch_bytes, sizeof(double) * 2 * (size_t)nb);
    cudaError_t e = launch_norms(a, b, count, prec, (double *)scratch, nb, out, (cudaStream_t)stream);
    return e == cudaSuccess ? LBM_OK : cuda_fail(e, "launching the norms kernels");
}

}  // extern "C"
