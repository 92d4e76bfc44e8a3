/*
 * Plain FP64 CPU oracle of the fully discrete finite-difference LB scheme.
 *
 * TEST INFRASTRUCTURE ONLY: only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark load this file; the CUDA library never does, and the two
 * share no code, header or table.
 *
 * What it computes (Ghiroldi & Gibelli, arXiv:1308.0692):
 *   - the discrete BGKW equation  d f_a/dt + xi_a . grad f_a = -(f_a - f^eq_a)/Kn   (Eq. 1)
 *     with f^eq_a = w_a rho (1 + xi_a . u) = w_a (rho + xi_a . j)                  (Eqs. 2-5)
 *     and rho = sum_a f_a, j = rho u = sum_a xi_a f_a                               (Eqs. 6-7);
 *   - Maxwell diffuse walls with complete accommodation, the re-emitted
 *     population being w_a rho_w (1 + xi_t U) for velocities leaving the wall  (Eq. 8),
 *     rho_w fixed by zero normal mass flux through the wall                      (Eq. 9);
 *   - the fully discrete scheme of the text after Table 2's figures: first-order
 *     time splitting of transport then relaxation, first-order upwind transport,
 *     explicit Euler relaxation.
 *
 * Readings of the paper fixed here (the CUDA path takes the same ones):
 *   - state: the perturbation h_a = (f_a - w_a) / u_ref, u_ref = max(|U_bottom|, |U_top|)
 *     (1 if both are zero); cold start h = 0 is f_a = w_a (rho = 1, u = 0);
 *   - grid: uniform, cell centred; walls lie on cell faces.  Couette: nx columns
 *     periodic in x, ny cells between plates at y = 0 (speed U_bottom) and
 *     y = 1 (speed U_top), square cells dx = dy = 1/ny.  Cavity: unit square,
 *     nx x ny cells, walls on all four faces; bottom moves at U_bottom, top at
 *     U_top (the lid), the side walls are at rest;
 *   - transport (dimensionally unsplit first-order upwind, finite-volume form):
 *       h*_a(c) = h_a(c) - nu_x,a [h_a(c) - h_a(c - s_x)] - nu_y,a [h_a(c) - h_a(c - s_y)]
 *     with nu_d,a = |xi_d,a| dt / dd and s_d = sign(xi_d,a); across a wall face
 *     the upwind value is the wall-emitted population (ghost) of that face;
 *   - ghost of face F for a velocity leaving the wall:
 *       h_a = w_a [ rho'_F (1 + xi_t,a U_F) + xi_t,a U_F / u_ref ],
 *       rho'_F = sum_{a: xi_a . n_F < 0} |xi_a . n_F| h_a(c) / D_F,
 *       D_F = sum_{a: xi_a . n_F > 0} (xi_a . n_F) w_a,
 *     n_F the unit normal into the gas, xi_t the tangential component, c the
 *     wall-adjacent cell at the current time level.  This is Eq. (8) with the
 *     discrete weight w_a in place of omega(xi_a), and Eq. (9) as a discrete flux
 *     balance; for the half-range sets D_F = 1/sqrt(2 pi) and it is Eq. (9)
 *     exactly, for full-range sets it keeps the wall impermeable;
 *   - relaxation: h^{n+1}_a = h*_a - omega (h*_a - w_a (rho' + xi_a . j')),
 *     omega = dt / Kn (0 for Kn = +inf), rho' = sum h*_a, j' = sum xi_a h*_a;
 *   - time step: dt = cfl / (max|xi_x|/dx + max|xi_y|/dy) (the x term dropped
 *     for a single periodic Couette column), then dt <= Kn;
 *   - residual: r = ||h^{n+1} - h^n||_2 / ||h^{n+1}||_2 over all cells and velocities.
 *
 * Layout: h[a * ncells + c], c = y * nx + x (structure of arrays), FP64.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

enum { ORC_COUETTE = 0, ORC_CAVITY = 1 };
enum { FACE_BOTTOM = 0, FACE_TOP = 1, FACE_LEFT = 2, FACE_RIGHT = 3 };

typedef struct {
    int n;              /* number of discrete velocities */
    const double *xi_x; /* [n] */
    const double *xi_y; /* [n] */
    const double *w;    /* [n] */
    int geom;           /* ORC_COUETTE or ORC_CAVITY */
    int nx, ny;
    double kn;          /* Knudsen number of Eq. (1); +inf = no collisions */
    double u_bottom, u_top;
    double cfl;
} orc_problem;

typedef struct {
    double dt, dx, dy, omega, u_ref;
    double d_x; /* sum over xi_x > 0 of xi_x w : wall-flux normaliser for x-normal faces */
    double d_y; /* sum over xi_y > 0 of xi_y w : same for y-normal faces */
} orc_coeffs;

int orc_coeffs_compute(const orc_problem *p, orc_coeffs *c)
{
    if (p->n <= 0 || p->nx <= 0 || p->ny <= 0 || !(p->kn > 0) || !(p->cfl > 0))
        return 1;
    double mx = 0, my = 0;
    c->d_x = 0;
    c->d_y = 0;
    for (int a = 0; a < p->n; ++a) {
        if (fabs(p->xi_x[a]) > mx) mx = fabs(p->xi_x[a]);
        if (fabs(p->xi_y[a]) > my) my = fabs(p->xi_y[a]);
        if (p->xi_x[a] > 0) c->d_x += p->xi_x[a] * p->w[a];
        if (p->xi_y[a] > 0) c->d_y += p->xi_y[a] * p->w[a];
    }
    if (p->geom == ORC_COUETTE) {
        c->dy = 1.0 / p->ny;
        c->dx = c->dy;
    } else {
        c->dx = 1.0 / p->nx;
        c->dy = 1.0 / p->ny;
    }
    double rate = my / c->dy;
    if (!(p->geom == ORC_COUETTE && p->nx == 1))
        rate += mx / c->dx;
    c->dt = p->cfl / rate;
    if (isfinite(p->kn) && c->dt > p->kn)
        c->dt = p->kn;
    c->omega = isfinite(p->kn) ? c->dt / p->kn : 0.0;
    double ub = fabs(p->u_bottom), ut = fabs(p->u_top);
    c->u_ref = ub > ut ? ub : ut;
    if (c->u_ref == 0) c->u_ref = 1.0;
    return 0;
}

/* rho'_F of Eq. (9) (discrete flux balance) for face F of cell `cell`. */
static double wall_density(const orc_problem *p, const orc_coeffs *c, const double *h,
                           long ncells, long cell, int face)
{
    double s = 0;
    for (int a = 0; a < p->n; ++a) {
        double xn; /* xi . n_F, n_F pointing into the gas */
        switch (face) {
        case FACE_BOTTOM: xn = p->xi_y[a]; break;
        case FACE_TOP:    xn = -p->xi_y[a]; break;
        case FACE_LEFT:   xn = p->xi_x[a]; break;
        default:          xn = -p->xi_x[a]; break;
        }
        if (xn < 0) s += -xn * h[(long)a * ncells + cell];
    }
    double d = (face == FACE_BOTTOM || face == FACE_TOP) ? c->d_y : c->d_x;
    return s / d;
}

/* Wall-emitted population of Eq. (8) in perturbation form, velocity a, face F. */
static double ghost(const orc_problem *p, const orc_coeffs *c, int face, int a, double rho_w)
{
    double xt, u;
    switch (face) {
    case FACE_BOTTOM: xt = p->xi_x[a]; u = p->u_bottom; break;
    case FACE_TOP:    xt = p->xi_x[a]; u = p->u_top; break;
    case FACE_LEFT:   xt = p->xi_y[a]; u = 0.0; break;
    default:          xt = p->xi_y[a]; u = 0.0; break;
    }
    return p->w[a] * (rho_w * (1.0 + xt * u) + xt * u / c->u_ref);
}

/* One time step at one cell: transport (upwind, walls) then relaxation; writes out[a], a < n. */
static void step_cell(const orc_problem *p, const orc_coeffs *c, const double *h, long cell,
                      double *hs, double *out)
{
    const int n = p->n, nx = p->nx, ny = p->ny;
    const long ncells = (long)nx * ny;
    const int x = (int)(cell % nx), y = (int)(cell / nx);
    const int cavity = p->geom == ORC_CAVITY;

    /* wall densities of the faces this cell touches (current time level) */
    double rho_b = 0, rho_t = 0, rho_l = 0, rho_r = 0;
    if (y == 0) rho_b = wall_density(p, c, h, ncells, cell, FACE_BOTTOM);
    if (y == ny - 1) rho_t = wall_density(p, c, h, ncells, cell, FACE_TOP);
    if (cavity && x == 0) rho_l = wall_density(p, c, h, ncells, cell, FACE_LEFT);
    if (cavity && x == nx - 1) rho_r = wall_density(p, c, h, ncells, cell, FACE_RIGHT);

    /* transport */
    for (int a = 0; a < n; ++a) {
        const double *ha = h + (long)a * ncells;
        double hc = ha[cell];
        double nux = fabs(p->xi_x[a]) * c->dt / c->dx;
        double nuy = fabs(p->xi_y[a]) * c->dt / c->dy;
        double hx = hc, hy = hc;
        if (p->xi_x[a] > 0) {
            if (x > 0) hx = ha[cell - 1];
            else if (cavity) hx = ghost(p, c, FACE_LEFT, a, rho_l);
            else hx = ha[cell + nx - 1];          /* periodic */
        } else if (p->xi_x[a] < 0) {
            if (x < nx - 1) hx = ha[cell + 1];
            else if (cavity) hx = ghost(p, c, FACE_RIGHT, a, rho_r);
            else hx = ha[cell - (nx - 1)];        /* periodic */
        }
        if (p->xi_y[a] > 0) {
            if (y > 0) hy = ha[cell - nx];
            else hy = ghost(p, c, FACE_BOTTOM, a, rho_b);
        } else if (p->xi_y[a] < 0) {
            if (y < ny - 1) hy = ha[cell + nx];
            else hy = ghost(p, c, FACE_TOP, a, rho_t);
        }
        hs[a] = hc - nux * (hc - hx) - nuy * (hc - hy);
    }

    /* moments of the transported populations (Eqs. 6-7) */
    double rho = 0, jx = 0, jy = 0;
    for (int a = 0; a < n; ++a) {
        rho += hs[a];
        jx += p->xi_x[a] * hs[a];
        jy += p->xi_y[a] * hs[a];
    }

    /* explicit Euler relaxation towards w_a (rho + xi_a . j) (Eqs. 1, 5) */
    for (int a = 0; a < n; ++a) {
        double heq = p->w[a] * (rho + p->xi_x[a] * jx + p->xi_y[a] * jy);
        out[a] = hs[a] - c->omega * (hs[a] - heq);
    }
}

/* Full step: h (SoA, n x ncells) -> hn. */
void orc_step(const orc_problem *p, const orc_coeffs *c, const double *h, double *hn)
{
    const long ncells = (long)p->nx * p->ny;
    const int n = p->n;
#pragma omp parallel
    {
        double *hs = (double *)malloc(sizeof(double) * n);
        double *out = (double *)malloc(sizeof(double) * n);
#pragma omp for schedule(static)
        for (long cell = 0; cell < ncells; ++cell) {
            step_cell(p, c, h, cell, hs, out);
            for (int a = 0; a < n; ++a) hn[(long)a * ncells + cell] = out[a];
        }
        free(hs);
        free(out);
    }
}

/*
 * Relaxation alone over a fraction of the time step: out_a = h_a - frac * omega *
 * (h_a - w_a (rho' + xi_a . j')) at every cell, with the moments of h (explicit Euler over
 * frac * dt).  With frac = 1/2 it is the half step of the symmetric (Strang) splitting
 * relaxation(dt/2) - transport(dt) - relaxation(dt/2), which the caller composes with
 * orc_step run on coefficients whose omega is halved.
 */
void orc_relax(const orc_problem *p, const orc_coeffs *c, const double *h, double *out, double frac)
{
    const long ncells = (long)p->nx * p->ny;
    const int n = p->n;
    const double om = frac * c->omega;
    for (long cell = 0; cell < ncells; ++cell) {
        double rho = 0, jx = 0, jy = 0;
        for (int a = 0; a < n; ++a) {
            const double v = h[(long)a * ncells + cell];
            rho += v;
            jx += p->xi_x[a] * v;
            jy += p->xi_y[a] * v;
        }
        for (int a = 0; a < n; ++a) {
            const double v = h[(long)a * ncells + cell];
            const double heq = p->w[a] * (rho + p->xi_x[a] * jx + p->xi_y[a] * jy);
            out[(long)a * ncells + cell] = v - om * (v - heq);
        }
    }
}

/*
 * Relaxation alone over frac * dt, exact for the linear relaxation equation:
 * out_a = E_a + exp(-frac * omega) (h_a - E_a), E_a = w_a (rho' + xi_a . j') (rho', j' of h,
 * which relaxation does not change).  Two of these over dt/2 make one over dt exactly.
 */
void orc_relax_exp(const orc_problem *p, const orc_coeffs *c, const double *h, double *out, double frac)
{
    const long ncells = (long)p->nx * p->ny;
    const int n = p->n;
    const double decay = exp(-frac * c->omega);
    for (long cell = 0; cell < ncells; ++cell) {
        double rho = 0, jx = 0, jy = 0;
        for (int a = 0; a < n; ++a) {
            const double v = h[(long)a * ncells + cell];
            rho += v;
            jx += p->xi_x[a] * v;
            jy += p->xi_y[a] * v;
        }
        for (int a = 0; a < n; ++a) {
            const double heq = p->w[a] * (rho + p->xi_x[a] * jx + p->xi_y[a] * jy);
            out[(long)a * ncells + cell] = heq + decay * (h[(long)a * ncells + cell] - heq);
        }
    }
}

/*
 * Second-order transport alone (an extension of the scheme, not the paper's first-order
 * upwind): finite-volume update h*_i = h_i - (F_out - F_in) per direction with the
 * upwind-biased second-order (Beam-Warming) face flux
 *     F = nu [h_u + (1 - nu)/2 (h_u - h_uu)],
 * h_u the upwind cell of the face and h_uu the next one upwind.  Where h_uu would lie beyond
 * a wall the face flux is first order, F = nu h_u; across a wall face the inflow is
 * nu times the wall-emitted population (Eq. 8).  The wall density of Eq. (9) balances the
 * outflow through the wall face as this flux computes it, i.e. it is formed from the face
 * values h_u + (1 - nu)/2 (h_u - h_uu) of the wall-adjacent cell (h_uu: the next cell
 * inward), so that the walls stay impermeable.  Periodic in x for Couette.
 */

/* h at (x, y) of velocity a, x periodic in Couette; caller keeps y in range */
static double hat(const orc_problem *p, const double *h, int a, int x, int y)
{
    const int nx = p->nx;
    if (p->geom == ORC_COUETTE) x = ((x % nx) + nx) % nx;
    return h[(long)a * nx * p->ny + (long)y * nx + x];
}

/* face value of the outflow through the wall face of wall-adjacent cell (x, y) for
 * velocity a moving towards the wall; (dx, dy) = step from the cell into the gas */
static double wall_face_value(const orc_problem *p, const double *h, int a, int x, int y, int dx, int dy,
                              double nu)
{
    const double hu = hat(p, h, a, x, y);
    const int xi = x + dx, yi = y + dy;
    if (xi < 0 || xi >= p->nx || yi < 0 || yi >= p->ny) return hu;   /* one-cell-wide domain */
    const double huu = hat(p, h, a, xi, yi);
    return hu + 0.5 * (1.0 - nu) * (hu - huu);
}

static double wall_density2(const orc_problem *p, const orc_coeffs *c, const double *h, int x, int y, int face)
{
    double s = 0;
    for (int a = 0; a < p->n; ++a) {
        double xn;
        int dx = 0, dy = 0;
        switch (face) {
        case FACE_BOTTOM: xn = p->xi_y[a]; dy = 1; break;
        case FACE_TOP:    xn = -p->xi_y[a]; dy = -1; break;
        case FACE_LEFT:   xn = p->xi_x[a]; dx = 1; break;
        default:          xn = -p->xi_x[a]; dx = -1; break;
        }
        if (xn < 0) {
            const double nu = -xn * c->dt / ((face == FACE_BOTTOM || face == FACE_TOP) ? c->dy : c->dx);
            s += -xn * wall_face_value(p, h, a, x, y, dx, dy, nu);
        }
    }
    return s / ((face == FACE_BOTTOM || face == FACE_TOP) ? c->d_y : c->d_x);
}

/* inflow/outflow fluxes along one axis for velocity a at cell position i (0..len-1) of
 * that axis, moving towards increasing index with Courant number nu; get(k) returns h at
 * index k of the axis (k may wrap if periodic); walls: ghost value g_lo at the low end */
static double flux_difference(double nu, int i, int len, int periodic, double g_lo, double (*get)(const void *, int),
                              const void *ctx)
{
    double fin, fout;
    const double hi = get(ctx, i);
    /* face i - 1/2 */
    if (!periodic && i == 0) {
        fin = nu * g_lo;
    } else {
        const double hu = get(ctx, i - 1);
        if (!periodic && i == 1) fin = nu * hu;
        else fin = nu * (hu + 0.5 * (1.0 - nu) * (hu - get(ctx, i - 2)));
    }
    /* face i + 1/2 */
    if (!periodic && i == 0) fout = nu * hi;
    else fout = nu * (hi + 0.5 * (1.0 - nu) * (hi - get(ctx, i - 1)));
    (void)len;
    return fout - fin;
}

typedef struct {
    const orc_problem *p;
    const double *h;
    int a, x, y, axis, dir;   /* axis 0: x, 1: y; dir +1: transport towards increasing index */
} axis_ctx;

/* h along the axis in transport order: index k counts from the upwind end */
static double axis_get(const void *v, int k)
{
    const axis_ctx *q = (const axis_ctx *)v;
    const int len = q->axis == 0 ? q->p->nx : q->p->ny;
    const int pos = q->dir > 0 ? k : len - 1 - k;
    return q->axis == 0 ? hat(q->p, q->h, q->a, pos, q->y) : hat(q->p, q->h, q->a, q->x, pos);
}

/* Second-order transport of every velocity at one cell: out[a * ostride], a < n. */
static void transport2_cell(const orc_problem *p, const orc_coeffs *c, const double *h, long cell, double *out,
                            long ostride)
{
    const int n = p->n, nx = p->nx, ny = p->ny;
    const long ncells = (long)nx * ny;
    const int cavity = p->geom == ORC_CAVITY;
    const int xmove = !(p->geom == ORC_COUETTE && nx == 1);
    const int x = (int)(cell % nx), y = (int)(cell / nx);
    double rho_b = 0, rho_t = 0, rho_l = 0, rho_r = 0;
    if (y == 0) rho_b = wall_density2(p, c, h, x, y, FACE_BOTTOM);
    if (y == ny - 1) rho_t = wall_density2(p, c, h, x, y, FACE_TOP);
    if (cavity && x == 0) rho_l = wall_density2(p, c, h, x, y, FACE_LEFT);
    if (cavity && x == nx - 1) rho_r = wall_density2(p, c, h, x, y, FACE_RIGHT);
    for (int a = 0; a < n; ++a) {
        double v = h[(long)a * ncells + cell];
        axis_ctx q = {p, h, a, x, y, 0, 1};
        if (xmove && p->xi_x[a] != 0) {
            const double nu = fabs(p->xi_x[a]) * c->dt / c->dx;
            q.axis = 0;
            q.dir = p->xi_x[a] > 0 ? 1 : -1;
            const int i = q.dir > 0 ? x : nx - 1 - x;
            const double g = cavity ? (q.dir > 0 ? ghost(p, c, FACE_LEFT, a, rho_l) : ghost(p, c, FACE_RIGHT, a, rho_r))
                                    : 0.0;
            v -= flux_difference(nu, i, nx, !cavity, g, axis_get, &q);
        }
        if (p->xi_y[a] != 0) {
            const double nu = fabs(p->xi_y[a]) * c->dt / c->dy;
            q.axis = 1;
            q.dir = p->xi_y[a] > 0 ? 1 : -1;
            const int i = q.dir > 0 ? y : ny - 1 - y;
            const double g = q.dir > 0 ? ghost(p, c, FACE_BOTTOM, a, rho_b) : ghost(p, c, FACE_TOP, a, rho_t);
            v -= flux_difference(nu, i, ny, 0, g, axis_get, &q);
        }
        out[(long)a * ostride] = v;
    }
}

void orc_transport2(const orc_problem *p, const orc_coeffs *c, const double *h, double *out)
{
    const long ncells = (long)p->nx * p->ny;
#pragma omp parallel for schedule(static)
    for (long cell = 0; cell < ncells; ++cell) transport2_cell(p, c, h, cell, out + cell, ncells);
}

/*
 * One step of the second-order variant in its stored-state form at selected cells only:
 * the second-order transport, then the exact relaxation over dt,
 * out = E + exp(-omega) (h* - E), E_a = w_a (rho' + xi_a . j') of h* -- the step that the
 * symmetric splitting with exact half relaxations takes on the half-relaxed state (as
 * orc_transport2 followed by orc_relax_exp with frac = 1).  out[k * n + a] for cells[k].
 */
void orc_step2_cells(const orc_problem *p, const orc_coeffs *c, const double *h, const long *cells,
                     long ncell_list, double *out)
{
    const int n = p->n;
    const double decay = exp(-c->omega);
    for (long k = 0; k < ncell_list; ++k) {
        double *o = out + k * n;
        transport2_cell(p, c, h, cells[k], o, 1);
        double rho = 0, jx = 0, jy = 0;
        for (int a = 0; a < n; ++a) {
            rho += o[a];
            jx += p->xi_x[a] * o[a];
            jy += p->xi_y[a] * o[a];
        }
        for (int a = 0; a < n; ++a) {
            const double heq = p->w[a] * (rho + p->xi_x[a] * jx + p->xi_y[a] * jy);
            o[a] = heq + decay * (o[a] - heq);
        }
    }
}

/* The step's result at selected cells only: out[k * n + a] for cells[k]. */
void orc_step_cells(const orc_problem *p, const orc_coeffs *c, const double *h,
                    const long *cells, long ncell_list, double *out)
{
    const int n = p->n;
    double *hs = (double *)malloc(sizeof(double) * n);
    for (long k = 0; k < ncell_list; ++k)
        step_cell(p, c, h, cells[k], hs, out + k * n);
    free(hs);
}

/* r = ||hn - h|| / ||hn|| (0 when both vanish); also returns the two squared norms. */
double orc_residual(const double *hn, const double *h, long count, double *sq_diff, double *sq_new)
{
    double sd = 0, sn = 0;
    for (long i = 0; i < count; ++i) {
        double d = hn[i] - h[i];
        sd += d * d;
        sn += hn[i] * hn[i];
    }
    if (sq_diff) *sq_diff = sd;
    if (sq_new) *sq_new = sn;
    if (sn == 0) return sd == 0 ? 0.0 : INFINITY;
    return sqrt(sd / sn);
}

/*
 * March from h (in place) until r < tol (checked every `every` steps) or max_steps.
 * Returns the steps taken; *r_out = the last residual evaluated (the step's change).
 */
long orc_march(const orc_problem *p, const orc_coeffs *c, double *h, long max_steps,
               long every, double tol, double *r_out)
{
    const long count = (long)p->n * p->nx * p->ny;
    double *tmp = (double *)malloc(sizeof(double) * count);
    double r = INFINITY;
    long s = 0;
    while (s < max_steps) {
        orc_step(p, c, h, tmp);
        ++s;
        if (every > 0 && (s % every == 0 || s == max_steps)) {
            r = orc_residual(tmp, h, count, NULL, NULL);
            memcpy(h, tmp, sizeof(double) * count);
            if (r < tol) break;
        } else {
            memcpy(h, tmp, sizeof(double) * count);
        }
    }
    free(tmp);
    if (r_out) *r_out = r;
    return s;
}

/*
 * Macroscopic fields in the units of Eq. (1) (linearised about rho = 1, u = 0):
 *   rho = 1 + u_ref sum h,  u = u_ref sum xi h / rho,
 *   P_ij = sum xi_i xi_j f = delta_ij + u_ref sum xi_i xi_j h  (sum w xi_i xi_j = delta_ij
 *   for every set used here).  Any output pointer may be NULL.
 */
void orc_moments(const orc_problem *p, const orc_coeffs *c, const double *h,
                 double *rho, double *ux, double *uy, double *pxx, double *pxy, double *pyy)
{
    const long ncells = (long)p->nx * p->ny;
    for (long cell = 0; cell < ncells; ++cell) {
        double s0 = 0, sx = 0, sy = 0, sxx = 0, sxy = 0, syy = 0;
        for (int a = 0; a < p->n; ++a) {
            double v = h[(long)a * ncells + cell];
            s0 += v;
            sx += p->xi_x[a] * v;
            sy += p->xi_y[a] * v;
            sxx += p->xi_x[a] * p->xi_x[a] * v;
            sxy += p->xi_x[a] * p->xi_y[a] * v;
            syy += p->xi_y[a] * p->xi_y[a] * v;
        }
        double r = 1.0 + c->u_ref * s0;
        if (rho) rho[cell] = r;
        if (ux) ux[cell] = c->u_ref * sx / r;
        if (uy) uy[cell] = c->u_ref * sy / r;
        if (pxx) pxx[cell] = 1.0 + c->u_ref * sxx;
        if (pxy) pxy[cell] = c->u_ref * sxy;
        if (pyy) pyy[cell] = 1.0 + c->u_ref * syy;
    }
}

/*
 * Momentum flux through the horizontal faces, p_xy = u_ref sum xi_x xi_y h_upwind,
 * the upwind value being the ghost on a wall face.  out[(j) * nx + x] for
 * faces j = 0..ny (j = 0 bottom wall, j = ny top wall).  This is the shear
 * stress the scheme actually transmits; at a steady Couette state it is the same
 * on every face.
 */
void orc_face_flux_y(const orc_problem *p, const orc_coeffs *c, const double *h, double *out)
{
    const int nx = p->nx, ny = p->ny;
    const long ncells = (long)nx * ny;
    for (int j = 0; j <= ny; ++j) {
        for (int x = 0; x < nx; ++x) {
            long below = (long)(j - 1) * nx + x, above = (long)j * nx + x;
            double rb = 0, rt = 0;
            if (j == 0) rb = wall_density(p, c, h, ncells, above, FACE_BOTTOM);
            if (j == ny) rt = wall_density(p, c, h, ncells, below, FACE_TOP);
            double s = 0;
            for (int a = 0; a < p->n; ++a) {
                double v;
                if (p->xi_y[a] > 0)
                    v = (j == 0) ? ghost(p, c, FACE_BOTTOM, a, rb) : h[(long)a * ncells + below];
                else if (p->xi_y[a] < 0)
                    v = (j == ny) ? ghost(p, c, FACE_TOP, a, rt) : h[(long)a * ncells + above];
                else
                    v = 0.0;
                s += p->xi_x[a] * p->xi_y[a] * v;
            }
            out[(long)j * nx + x] = c->u_ref * s;
        }
    }
}

/* Same through the vertical faces (y-momentum flux p_yx), out[y * (nx+1) + i], i = 0..nx;
 * cavity only (faces i = 0 and i = nx are the side walls). */
void orc_face_flux_x(const orc_problem *p, const orc_coeffs *c, const double *h, double *out)
{
    const int nx = p->nx, ny = p->ny;
    const long ncells = (long)nx * ny;
    for (int y = 0; y < ny; ++y) {
        for (int i = 0; i <= nx; ++i) {
            long left = (long)y * nx + i - 1, right = (long)y * nx + i;
            double rl = 0, rr = 0;
            if (i == 0) rl = wall_density(p, c, h, ncells, right, FACE_LEFT);
            if (i == nx) rr = wall_density(p, c, h, ncells, left, FACE_RIGHT);
            double s = 0;
            for (int a = 0; a < p->n; ++a) {
                double v;
                if (p->xi_x[a] > 0)
                    v = (i == 0) ? ghost(p, c, FACE_LEFT, a, rl) : h[(long)a * ncells + left];
                else if (p->xi_x[a] < 0)
                    v = (i == nx) ? ghost(p, c, FACE_RIGHT, a, rr) : h[(long)a * ncells + right];
                else
                    v = 0.0;
                s += p->xi_x[a] * p->xi_y[a] * v;
            }
            out[(long)y * (nx + 1) + i] = c->u_ref * s;
        }
    }
}

/*
 * Momentum fluxes through the cell faces for the second-order transport: the upwind face
 * value of orc_transport2 (second-order reconstruction, first order where the next upwind
 * cell lies beyond a wall, the wall-emitted population on a wall face), weighted by
 * xi_x xi_y.  At a steady state this flux is the same through every face of a Couette
 * channel.  Layout as orc_face_flux_y / orc_face_flux_x.
 */
static double face_value2(const orc_problem *p, const orc_coeffs *c, const double *h, int a, int axis,
                          int x, int y, int j, double rho_lo, double rho_hi)
{
    /* face j on `axis` between cells j-1 and j of the line through (x, y); j = 0..len */
    const int len = axis == 0 ? p->nx : p->ny;
    const double xi = axis == 0 ? p->xi_x[a] : p->xi_y[a];
    const double nu = fabs(xi) * c->dt / (axis == 0 ? c->dx : c->dy);
    const int periodic = axis == 0 && p->geom == ORC_COUETTE;
#define H_AT(k) (axis == 0 ? hat(p, h, a, (k), y) : hat(p, h, a, x, (k)))
    if (xi > 0) {
        if (!periodic && j == 0)
            return ghost(p, c, axis == 0 ? FACE_LEFT : FACE_BOTTOM, a, rho_lo);
        const double hu = H_AT(j - 1);
        if (!periodic && j == 1) return hu;
        return hu + 0.5 * (1.0 - nu) * (hu - H_AT(j - 2));
    }
    if (xi < 0) {
        if (!periodic && j == len)
            return ghost(p, c, axis == 0 ? FACE_RIGHT : FACE_TOP, a, rho_hi);
        const double hu = H_AT(j);
        if (!periodic && j == len - 1) return hu;
        return hu + 0.5 * (1.0 - nu) * (hu - H_AT(j + 1));
    }
#undef H_AT
    return 0.0;
}

void orc_face_flux2_y(const orc_problem *p, const orc_coeffs *c, const double *h, double *out)
{
    const int nx = p->nx, ny = p->ny;
    for (int x = 0; x < nx; ++x) {
        const double rb = wall_density2(p, c, h, x, 0, FACE_BOTTOM);
        const double rt = wall_density2(p, c, h, x, ny - 1, FACE_TOP);
        for (int j = 0; j <= ny; ++j) {
            double s = 0;
            for (int a = 0; a < p->n; ++a)
                s += p->xi_x[a] * p->xi_y[a] * face_value2(p, c, h, a, 1, x, 0, j, rb, rt);
            out[(long)j * nx + x] = c->u_ref * s;
        }
    }
}

void orc_face_flux2_x(const orc_problem *p, const orc_coeffs *c, const double *h, double *out)
{
    const int nx = p->nx, ny = p->ny;
    for (int y = 0; y < ny; ++y) {
        const double rl = wall_density2(p, c, h, 0, y, FACE_LEFT);
        const double rr = wall_density2(p, c, h, nx - 1, y, FACE_RIGHT);
        for (int i = 0; i <= nx; ++i) {
            double s = 0;
            for (int a = 0; a < p->n; ++a)
                s += p->xi_x[a] * p->xi_y[a] * face_value2(p, c, h, a, 0, 0, y, i, rl, rr);
            out[(long)y * (nx + 1) + i] = c->u_ref * s;
        }
    }
}
