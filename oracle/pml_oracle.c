/*
 * Plain FP64 CPU oracle for the reflectionless discrete PML (Chern, arXiv 1804.01390).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / reference legs may load this code.  It shares no source with the
 * CUDA library (paper_1804_01390_gb300/csrc) and the library never calls it.
 *
 * Everything here is written to be checked against the paper by eye:
 *   - semi-discrete operator A of eq:DiscretePML (Sec. 1.1.2, Eq. 3a-3c), evaluated
 *     vertex by vertex with periodic index wrap (the paper truncates the layer with a
 *     periodic box, Sec. 1.1.3);
 *   - classic four-stage Runge-Kutta (Sec. 1.1.3 names RK4), stage by stage;
 *   - the spring-mass energy eq:Energy (Sec. 1.1.5);
 *   - the discrete adjoint of one RK4 step (reverse of the stage graph, with the
 *     transpose of A written out from the entries of A).
 * Compiled with -O2 -ffp-contract=off so every product and sum is rounded once, in
 * source order.
 *
 * Conventions (readings of the paper where it leaves a choice open):
 *   - axis a has T[a] vertices 0..T[a]-1, periodic; the physical vertices are
 *     w..w+N-1 and the layer vertices the other 2w;
 *   - sigma_a[e] is edge-centred: it belongs to the edge (e, e+1 mod T) - this is the
 *     placement of s_j in eq:VertexPositions and of sigma(j) in eq:IntroSolution;
 *   - Phi_a is supported where sigma_a[i_a] != 0 and Psi_a where sigma_a[i_a - 1] != 0
 *     (Sec. 1.1.2, the support statement after Eq. 3); elsewhere they are held at 0.
 *     Outside that support they only ever appear multiplied by a zero sigma.
 *
 * State layout: one contiguous array of nf = 2 + 2*ndim fields of n = T0*T1*T2
 * doubles: [U, V, Phi_0, Psi_0, Phi_1, Psi_1, Phi_2, Psi_2]; vertex (x, y, z) sits at
 * flat index x + T0*(y + T1*z).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846

typedef struct {
    int ndim;
    int64_t T[3];
    double h;
    const double *sig[3];
    int wall;            /* 0: periodic box; 1: every field is zero beyond both ends of every axis */
} orc_grid;

/*
 * Boundary of the box for the calls that follow: 0 periodic (the paper's truncation,
 * Sec. 1.1.3), 1 a reflecting wall just beyond each end (the layer backed by a reflecting
 * boundary of Sec. 1.1.4: U, V, Phi, Psi are zero at the vertices -1 and T; the caller's
 * sigma has sigma[T-1] = 0, there being no edge from T-1 to 0).
 */
static int g_wall = 0;
void orc_set_boundary(int wall) { g_wall = wall ? 1 : 0; }

typedef struct {
    int ns;
    const int64_t *idx;  /* flat vertex index of each source */
    const double *amp;   /* amplitude a_s */
    double f_peak;       /* Ricker peak frequency (1/time) */
    double t_delay;      /* Ricker centre time */
} orc_src;

static void grid_from_args(orc_grid *g, int ndim, const int64_t *T, double h, const double *sig_concat)
{
    int a;
    g->ndim = ndim;
    g->h = h;
    g->wall = g_wall;
    for (a = 0; a < 3; a++) g->T[a] = (a < ndim) ? T[a] : 1;
    {
        const double *p = sig_concat;
        for (a = 0; a < 3; a++) {
            g->sig[a] = (a < ndim) ? p : NULL;
            if (a < ndim) p += g->T[a];
        }
    }
}

static int64_t grid_n(const orc_grid *g) { return g->T[0] * g->T[1] * g->T[2]; }

static void to_coords(const orc_grid *g, int64_t i, int64_t c[3])
{
    c[0] = i % g->T[0];
    c[1] = (i / g->T[0]) % g->T[1];
    c[2] = i / (g->T[0] * g->T[1]);
}

static int64_t to_flat(const orc_grid *g, const int64_t c[3])
{
    return c[0] + g->T[0] * (c[1] + g->T[1] * c[2]);
}

/* flat index of the vertex c + s*e_a, wrapping periodically along axis a; with a wall,
 * -1 for a vertex beyond the end of the box (read as zero through at()) */
static int64_t shifted(const orc_grid *g, const int64_t c[3], int a, int s)
{
    int64_t d[3];
    d[0] = c[0]; d[1] = c[1]; d[2] = c[2];
    if (g->wall && (d[a] + s < 0 || d[a] + s >= g->T[a])) return -1;
    d[a] = ((d[a] + s) % g->T[a] + g->T[a]) % g->T[a];
    return to_flat(g, d);
}

static double at(const double *f, int64_t i) { return i < 0 ? 0.0 : f[i]; }

/* Ricker time function g(t) = (1 - 2 pi^2 f^2 (t-t0)^2) exp(-pi^2 f^2 (t-t0)^2). */
double orc_ricker(double t, double f_peak, double t_delay)
{
    double a = ORC_PI * ORC_PI * f_peak * f_peak * (t - t_delay) * (t - t_delay);
    return (1.0 - 2.0 * a) * exp(-a);
}

/*
 * Damping profile along one axis (edge-centred, length T = N + 2w).
 * d_e = max(a-1-e, e-b, 0) with a = w, b = w+N-1 is the depth of edge e in the
 * layer (0 on the physical edges and on the two interface edges, w on the wrap edge).
 *   kind 0: constant  sigma_max * [d_e > 0]               (paper Fig. HalfSpaceGauss)
 *   kind 1: power law sigma_max * (d_e / w)^order        (quadratic ramp: order 2)
 *   kind 2: random    sigma_max * u_e * [d_e > 0], u_e = draws[e] in [0,1)
 *                                                        (paper Fig. HalfSpaceRand)
 * Returns 0, or -1 on bad arguments.
 */
int orc_sigma_profile(int64_t N, int64_t w, int kind, double sigma_max, double order,
                      const double *draws, double *out)
{
    int64_t T = N + 2 * w, e;
    int64_t a = w, b = w + N - 1;
    if (N < 1 || w < 0) return -1;
    for (e = 0; e < T; e++) {
        int64_t d = 0;
        if (a - 1 - e > d) d = a - 1 - e;
        if (e - b > d) d = e - b;
        if (d == 0) { out[e] = 0.0; continue; }
        if (kind == 0) out[e] = sigma_max;
        else if (kind == 1) out[e] = sigma_max * pow((double)d / (double)w, order);
        else if (kind == 2) out[e] = sigma_max * draws[e];
        else return -1;
    }
    return 0;
}

/*
 * Integer layout tables along one axis of length T (bit-exact reference for the
 * library's own tables):
 *   phi_active[i] = sigma[i] != 0              (support of Phi, Sec. 1.1.2)
 *   psi_active[i] = sigma[i-1 mod T] != 0      (support of Psi)
 *   interior[i]   = 1 when the damping on the four edges i-2, i-1, i, i+1 is zero,
 *                   i.e. no PML term enters the V equation at i-1, i or i+1, and i
 *                   belongs to the contiguous run of such vertices that contains
 *                   the vertex `centre`.  On such vertices one RK4 step of Eq. 3
 *                   reduces exactly to one RK4 step of eq:DiscreteWaveEquation.
 */
void orc_layout_axis(const double *sig, int64_t T, int64_t centre,
                     uint8_t *phi_active, uint8_t *psi_active, uint8_t *interior)
{
    int64_t i, k;
    uint8_t *free4 = (uint8_t *)malloc((size_t)T);
    for (i = 0; i < T; i++) {
        phi_active[i] = (uint8_t)(sig[i] != 0.0);
        psi_active[i] = (uint8_t)(sig[(i - 1 + T) % T] != 0.0);
        interior[i] = 0;
    }
    for (i = 0; i < T; i++) {
        int ok = 1;
        for (k = -2; k <= 1; k++)
            if (sig[((i + k) % T + T) % T] != 0.0) ok = 0;
        free4[i] = (uint8_t)ok;
    }
    if (free4[centre]) {
        int64_t lo = centre, hi = centre, steps = 0;
        while (steps < T - 1 && free4[(lo - 1 + T) % T]) { lo--; steps++; }
        while (steps < T - 1 && free4[(hi + 1) % T]) { hi++; steps++; }
        for (i = lo; i <= hi; i++) interior[(i % T + T) % T] = 1;
    }
    free(free4);
}

/*
 * out = A y + b(t): the right-hand side of eq:DiscretePML (Eq. 3a-3c) in first-order
 * form with V = dU/dt:
 *   dU/dt   = V
 *   dV/dt   = sum_a (U(i+e_a) - 2U(i) + U(i-e_a))/h^2
 *           + sum_a (sigma_a[i_a] Psi_a(i+e_a) - sigma_a[i_a-1] Phi_a(i-e_a))/h   (+ sources)
 *   dPhi_a/dt = -1/2 (sigma_a[i_a-1] Phi_a(i-e_a) + sigma_a[i_a] Phi_a(i))
 *               - (U(i+e_a) - U(i-e_a))/(2h)        where sigma_a[i_a]   != 0, else 0
 *   dPsi_a/dt = -1/2 (sigma_a[i_a-1] Psi_a(i) + sigma_a[i_a] Psi_a(i+e_a))
 *               - (U(i+e_a) - U(i-e_a))/(2h)        where sigma_a[i_a-1] != 0, else 0
 * Sources add amp_s * g(t) to dV/dt at their vertex.
 */
static void rhs(const orc_grid *g, const double *y, double *out, const orc_src *src, double t)
{
    const int64_t n = grid_n(g);
    const double h = g->h;
    const double *U = y, *V = y + n;
    double *oU = out, *oV = out + n;
    int64_t i;
#pragma omp parallel for schedule(static)
    for (i = 0; i < n; i++) {
        int64_t c[3];
        int a;
        double lap = 0.0, pml = 0.0;
        to_coords(g, i, c);
        oU[i] = V[i];
        for (a = 0; a < g->ndim; a++) {
            int64_t ip = shifted(g, c, a, +1), im = shifted(g, c, a, -1);
            lap += (at(U, ip) - 2.0 * U[i] + at(U, im)) / (h * h);
        }
        for (a = 0; a < g->ndim; a++) {
            const double *Phi = y + (2 + 2 * a) * n, *Psi = y + (3 + 2 * a) * n;
            double *oPhi = out + (2 + 2 * a) * n, *oPsi = out + (3 + 2 * a) * n;
            const int64_t Ta = g->T[a];
            const double s_i = g->sig[a][c[a]];
            const double s_im = g->sig[a][(c[a] - 1 + Ta) % Ta];
            int64_t ip = shifted(g, c, a, +1), im = shifted(g, c, a, -1);
            double dU = (at(U, ip) - at(U, im)) / (2.0 * h);
            pml += (s_i * at(Psi, ip) - s_im * at(Phi, im)) / h;
            oPhi[i] = (s_i != 0.0) ? -0.5 * (s_im * at(Phi, im) + s_i * Phi[i]) - dU : 0.0;
            oPsi[i] = (s_im != 0.0) ? -0.5 * (s_im * Psi[i] + s_i * at(Psi, ip)) - dU : 0.0;
        }
        oV[i] = lap + pml;
    }
    if (src) {
        int s;
        for (s = 0; s < src->ns; s++)
            oV[src->idx[s]] += src->amp[s] * orc_ricker(t, src->f_peak, src->t_delay);
    }
}

/* Public single evaluation of A y (+ b(t) when src_ns > 0). */
void orc_rhs(int ndim, const int64_t *T, double h, const double *sig, const double *y, double *out,
             int src_ns, const int64_t *src_idx, const double *src_amp, double f_peak, double t_delay,
             double t)
{
    orc_grid g;
    orc_src s;
    grid_from_args(&g, ndim, T, h, sig);
    s.ns = src_ns; s.idx = src_idx; s.amp = src_amp; s.f_peak = f_peak; s.t_delay = t_delay;
    rhs(&g, y, out, src_ns > 0 ? &s : NULL, t);
}

/*
 * nsteps classic RK4 steps of dy/dt = A y + b(t) (Sec. 1.1.3), starting at step index
 * step0 (time t = step0*dt).  Butcher tableau c = (0, 1/2, 1/2, 1),
 * b = (1/6, 1/3, 1/3, 1/6).  When nr > 0, trace[k*nr + r] receives U at receiver r
 * after step k+1.  Returns 0, or -1 when scratch cannot be allocated.
 */
int orc_rk4(int ndim, const int64_t *T, double h, const double *sig, double *y, int64_t nsteps,
            double dt, int64_t step0, int src_ns, const int64_t *src_idx, const double *src_amp,
            double f_peak, double t_delay, int nr, const int64_t *rec_idx, double *trace)
{
    orc_grid g;
    orc_src s;
    int64_t n, len, k, j;
    double *k1, *k2, *k3, *k4, *Y;
    grid_from_args(&g, ndim, T, h, sig);
    s.ns = src_ns; s.idx = src_idx; s.amp = src_amp; s.f_peak = f_peak; s.t_delay = t_delay;
    n = grid_n(&g);
    len = (2 + 2 * (int64_t)ndim) * n;
    k1 = (double *)malloc(sizeof(double) * (size_t)len);
    k2 = (double *)malloc(sizeof(double) * (size_t)len);
    k3 = (double *)malloc(sizeof(double) * (size_t)len);
    k4 = (double *)malloc(sizeof(double) * (size_t)len);
    Y = (double *)malloc(sizeof(double) * (size_t)len);
    if (!k1 || !k2 || !k3 || !k4 || !Y) {
        free(k1); free(k2); free(k3); free(k4); free(Y);
        return -1;
    }
    for (k = 0; k < nsteps; k++) {
        const double t = (double)(step0 + k) * dt;
        const orc_src *sp = src_ns > 0 ? &s : NULL;
        rhs(&g, y, k1, sp, t);
#pragma omp parallel for schedule(static)
        for (j = 0; j < len; j++) Y[j] = y[j] + 0.5 * dt * k1[j];
        rhs(&g, Y, k2, sp, t + 0.5 * dt);
#pragma omp parallel for schedule(static)
        for (j = 0; j < len; j++) Y[j] = y[j] + 0.5 * dt * k2[j];
        rhs(&g, Y, k3, sp, t + 0.5 * dt);
#pragma omp parallel for schedule(static)
        for (j = 0; j < len; j++) Y[j] = y[j] + dt * k3[j];
        rhs(&g, Y, k4, sp, t + dt);
#pragma omp parallel for schedule(static)
        for (j = 0; j < len; j++)
            y[j] = y[j] + dt / 6.0 * (k1[j] + 2.0 * k2[j] + 2.0 * k3[j] + k4[j]);
        if (nr > 0) {
            int r;
            for (r = 0; r < nr; r++) trace[k * nr + r] = y[rec_idx[r]];
        }
    }
    free(k1); free(k2); free(k3); free(k4); free(Y);
    return 0;
}

/*
 * Spring-mass energy eq:Energy (Sec. 1.1.5):
 *   E = 1/2 sum_i V(i)^2 + 1/2 sum_i sum_a ((U(i+e_a) - U(i))/h)^2
 * with i over the box lo[a] <= i_a <= hi[a] (inclusive; the physical window).  The
 * forward difference at the last window vertex reads the next vertex, which may lie
 * in the layer (or wrap around when the window is the whole periodic box).
 */
double orc_energy(int ndim, const int64_t *T, double h, const double *y, const int64_t *lo,
                  const int64_t *hi)
{
    orc_grid g;
    int64_t n, i;
    double kin = 0.0, ela = 0.0;
    g.ndim = ndim; g.h = h; g.wall = g_wall;
    g.T[0] = T[0]; g.T[1] = ndim > 1 ? T[1] : 1; g.T[2] = ndim > 2 ? T[2] : 1;
    g.sig[0] = g.sig[1] = g.sig[2] = NULL;
    n = grid_n(&g);
    for (i = 0; i < n; i++) {
        int64_t c[3];
        int a, inside = 1;
        to_coords(&g, i, c);
        for (a = 0; a < ndim; a++)
            if (c[a] < lo[a] || c[a] > hi[a]) inside = 0;
        if (!inside) continue;
        kin += y[n + i] * y[n + i];
        for (a = 0; a < ndim; a++) {
            double d = (at(y, shifted(&g, c, a, +1)) - y[i]) / h;
            ela += d * d;
        }
    }
    return 0.5 * kin + 0.5 * ela;
}

/*
 * Norms of field U over the inclusive window lo..hi: out[0] = max |U|,
 * out[1] = sqrt(sum U^2), out[2] = sqrt(sum (U - ref)^2) (0 when ref is NULL).
 */
void orc_norms(int ndim, const int64_t *T, const double *U, const double *ref, const int64_t *lo,
               const int64_t *hi, double *out)
{
    orc_grid g;
    int64_t n, i;
    double mx = 0.0, s2 = 0.0, d2 = 0.0;
    g.ndim = ndim; g.h = 1.0;
    g.T[0] = T[0]; g.T[1] = ndim > 1 ? T[1] : 1; g.T[2] = ndim > 2 ? T[2] : 1;
    n = grid_n(&g);
    for (i = 0; i < n; i++) {
        int64_t c[3];
        int a, inside = 1;
        to_coords(&g, i, c);
        for (a = 0; a < ndim; a++)
            if (c[a] < lo[a] || c[a] > hi[a]) inside = 0;
        if (!inside) continue;
        if (fabs(U[i]) > mx) mx = fabs(U[i]);
        s2 += U[i] * U[i];
        if (ref) d2 += (U[i] - ref[i]) * (U[i] - ref[i]);
    }
    out[0] = mx; out[1] = sqrt(s2); out[2] = sqrt(d2);
}

/*
 * out = A^T ybar: the transpose of the operator in rhs(), collected entry by entry
 * (every coefficient A[r][c] of rhs() contributes A[r][c]*ybar[r] to out[c]):
 *   (A^T ybar)_U(i)   = sum_a (Vb(i+e) - 2Vb(i) + Vb(i-e))/h^2
 *                      + sum_a (Phib_a(i+e) - Phib_a(i-e))/(2h) + (Psib_a(i+e) - Psib_a(i-e))/(2h)
 *   (A^T ybar)_V(i)   = Ub(i)
 *   (A^T ybar)_Phi(i) = -sigma[i] Vb(i+e)/h - 1/2 sigma[i] (Phib(i+e) + Phib(i))
 *   (A^T ybar)_Psi(i) = +sigma[i-1] Vb(i-e)/h - 1/2 sigma[i-1] (Psib(i) + Psib(i-e))
 * Phib/Psib are first restricted to the supports (the rows of A outside the support
 * are zero), so the U row only sees supported entries.
 */
static void rhs_transpose(const orc_grid *g, const double *yb, double *out)
{
    const int64_t n = grid_n(g);
    const double h = g->h;
    const double *Ub = yb, *Vb = yb + n;
    int64_t i;
#pragma omp parallel for schedule(static)
    for (i = 0; i < n; i++) {
        int64_t c[3];
        int a;
        double acc = 0.0;
        to_coords(g, i, c);
        out[n + i] = Ub[i];
        for (a = 0; a < g->ndim; a++) {
            int64_t ip = shifted(g, c, a, +1), im = shifted(g, c, a, -1);
            acc += (at(Vb, ip) - 2.0 * Vb[i] + at(Vb, im)) / (h * h);
        }
        for (a = 0; a < g->ndim; a++) {
            const double *Phib = yb + (2 + 2 * a) * n, *Psib = yb + (3 + 2 * a) * n;
            double *oPhi = out + (2 + 2 * a) * n, *oPsi = out + (3 + 2 * a) * n;
            const int64_t Ta = g->T[a];
            const int64_t ia = c[a];
            const int64_t iap = (ia + 1) % Ta, iam = (ia - 1 + Ta) % Ta, iamm = (ia - 2 + Ta) % Ta;
            const double s_i = g->sig[a][ia], s_im = g->sig[a][iam];
            int64_t ip = shifted(g, c, a, +1), im = shifted(g, c, a, -1);
            /* supported adjoint entries (Phi support: sigma[j] != 0; Psi: sigma[j-1] != 0) */
            double phib_p = (g->sig[a][iap] != 0.0) ? at(Phib, ip) : 0.0;
            double phib_m = (g->sig[a][iam] != 0.0) ? at(Phib, im) : 0.0;
            double phib_0 = (s_i != 0.0) ? Phib[i] : 0.0;
            double psib_p = (s_i != 0.0) ? at(Psib, ip) : 0.0;        /* support of Psi(i+1): sigma[i] */
            double psib_m = (g->sig[a][iamm] != 0.0) ? at(Psib, im) : 0.0; /* Psi(i-1): sigma[i-2] */
            double psib_0 = (s_im != 0.0) ? Psib[i] : 0.0;
            acc += (phib_p - phib_m) / (2.0 * h) + (psib_p - psib_m) / (2.0 * h);
            oPhi[i] = (s_i != 0.0) ? -s_i * at(Vb, ip) / h - 0.5 * s_i * (phib_p + phib_0) : 0.0;
            oPsi[i] = (s_im != 0.0) ? s_im * at(Vb, im) / h - 0.5 * s_im * (psib_0 + psib_m) : 0.0;
        }
        out[i] = acc;
    }
}

void orc_rhs_transpose(int ndim, const int64_t *T, double h, const double *sig, const double *yb,
                       double *out)
{
    orc_grid g;
    grid_from_args(&g, ndim, T, h, sig);
    rhs_transpose(&g, yb, out);
}

/*
 * Discrete adjoint of nsteps RK4 steps, run backwards from step index step_end.
 * For k = 0..nsteps-1 the forward state index is m = step_end - k:
 *   1. ybar_U(x_r) += residual[k*nr + r]   (dJ/dU_m at the receivers)
 *   2. reverse the RK4 step m-1 -> m (times t = (m-1)dt, t+dt/2, t+dt):
 *        kb1 = dt/6 yb, kb2 = dt/3 yb, kb3 = dt/3 yb, kb4 = dt/6 yb
 *        Y4b = A^T kb4;  yb += Y4b;  kb3 += dt   * Y4b
 *        Y3b = A^T kb3;  yb += Y3b;  kb2 += dt/2 * Y3b
 *        Y2b = A^T kb2;  yb += Y2b;  kb1 += dt/2 * Y2b
 *        Y1b = A^T kb1;  yb += Y1b
 *      and for each source: grad_amp[s] += g(t) kb1_V + g(t+dt/2) (kb2_V + kb3_V)
 *                                          + g(t+dt) kb4_V  at x_s.
 * yb holds dJ/dy_{step_end} on entry and dJ/dy_{step_end - nsteps} on exit.
 * Returns 0, or -1 when scratch cannot be allocated.
 */
int orc_adjoint(int ndim, const int64_t *T, double h, const double *sig, double *yb,
                int64_t nsteps, double dt, int64_t step_end, int src_ns, const int64_t *src_idx,
                double f_peak, double t_delay, double *grad_amp, int nr, const int64_t *rec_idx,
                const double *residual)
{
    orc_grid g;
    int64_t n, len, k, j;
    double *kb1, *kb2, *kb3, *kb4, *Yb, *yb_out;
    grid_from_args(&g, ndim, T, h, sig);
    n = grid_n(&g);
    len = (2 + 2 * (int64_t)ndim) * n;
    kb1 = (double *)malloc(sizeof(double) * (size_t)len);
    kb2 = (double *)malloc(sizeof(double) * (size_t)len);
    kb3 = (double *)malloc(sizeof(double) * (size_t)len);
    kb4 = (double *)malloc(sizeof(double) * (size_t)len);
    Yb = (double *)malloc(sizeof(double) * (size_t)len);
    yb_out = (double *)malloc(sizeof(double) * (size_t)len);
    if (!kb1 || !kb2 || !kb3 || !kb4 || !Yb || !yb_out) {
        free(kb1); free(kb2); free(kb3); free(kb4); free(Yb); free(yb_out);
        return -1;
    }
    for (k = 0; k < nsteps; k++) {
        const int64_t m = step_end - k;
        const double t = (double)(m - 1) * dt;
        if (nr > 0) {
            int r;
            for (r = 0; r < nr; r++) yb[rec_idx[r]] += residual[k * nr + r];
        }
        for (j = 0; j < len; j++) {
            kb1[j] = dt / 6.0 * yb[j];
            kb2[j] = dt / 3.0 * yb[j];
            kb3[j] = dt / 3.0 * yb[j];
            kb4[j] = dt / 6.0 * yb[j];
            yb_out[j] = yb[j];
        }
        rhs_transpose(&g, kb4, Yb);
        for (j = 0; j < len; j++) { yb_out[j] += Yb[j]; kb3[j] += dt * Yb[j]; }
        rhs_transpose(&g, kb3, Yb);
        for (j = 0; j < len; j++) { yb_out[j] += Yb[j]; kb2[j] += 0.5 * dt * Yb[j]; }
        rhs_transpose(&g, kb2, Yb);
        for (j = 0; j < len; j++) { yb_out[j] += Yb[j]; kb1[j] += 0.5 * dt * Yb[j]; }
        rhs_transpose(&g, kb1, Yb);
        for (j = 0; j < len; j++) yb_out[j] += Yb[j];
        if (src_ns > 0 && grad_amp) {
            int s;
            for (s = 0; s < src_ns; s++) {
                const int64_t v = n + src_idx[s];
                grad_amp[s] += orc_ricker(t, f_peak, t_delay) * kb1[v]
                             + orc_ricker(t + 0.5 * dt, f_peak, t_delay) * (kb2[v] + kb3[v])
                             + orc_ricker(t + dt, f_peak, t_delay) * kb4[v];
            }
        }
        memcpy(yb, yb_out, sizeof(double) * (size_t)len);
    }
    free(kb1); free(kb2); free(kb3); free(kb4); free(Yb); free(yb_out);
    return 0;
}

/*
 * k^T (dA/dsigma_a[e]) Y for one edge e of axis a (sigma_a[e] != 0), with the supports of
 * Phi/Psi held fixed.  Written out from the sigma entries of eq:DiscretePML:
 *   dV/dt(i)     has  sigma_a[i_a] Psi_a(i+e_a)/h  and  -sigma_a[i_a-1] Phi_a(i-e_a)/h
 *   dPhi_a/dt(i) has -sigma_a[i_a-1] Phi_a(i-e_a)/2 and -sigma_a[i_a] Phi_a(i)/2   (if sigma_a[i_a] != 0)
 *   dPsi_a/dt(i) has -sigma_a[i_a-1] Psi_a(i)/2     and -sigma_a[i_a] Psi_a(i+e_a)/2 (if sigma_a[i_a-1] != 0)
 * so the vertices with i_a = e (sigma_a[i_a]) and i_a = e+1 (sigma_a[i_a-1]) contribute.
 */
static double dA_contract(const orc_grid *g, int a, int64_t e, const double *kb, const double *Y)
{
    const int64_t n = grid_n(g), Ta = g->T[a];
    const double h = g->h;
    const double *kV = kb + n, *kPhi = kb + (2 + 2 * a) * n, *kPsi = kb + (3 + 2 * a) * n;
    const double *Phi = Y + (2 + 2 * a) * n, *Psi = Y + (3 + 2 * a) * n;
    const int psi_at_e = g->sig[a][(e - 1 + Ta) % Ta] != 0.0;   /* Psi row active at i_a = e   */
    const int phi_at_e1 = g->sig[a][(e + 1) % Ta] != 0.0;       /* Phi row active at i_a = e+1 */
    double sum = 0.0;
    int64_t i;
    for (i = 0; i < n; i++) {
        int64_t c[3];
        to_coords(g, i, c);
        if (c[a] == e) {
            const int64_t ip = shifted(g, c, a, +1);
            sum += kV[i] * at(Psi, ip) / h;
            sum += -0.5 * kPhi[i] * Phi[i];
            if (psi_at_e) sum += -0.5 * kPsi[i] * at(Psi, ip);
        } else if (c[a] == (e + 1) % Ta) {
            const int64_t im = shifted(g, c, a, -1);
            sum += -kV[i] * at(Phi, im) / h;
            if (phi_at_e1) sum += -0.5 * kPhi[i] * at(Phi, im);
            sum += -0.5 * kPsi[i] * Psi[i];
        }
    }
    return sum;
}

/*
 * Misfit J = 1/2 sum_{m=1..nsteps} sum_r (U_m(x_r) - target[(m-1)*nr + r])^2 of the RK4 run
 * from y0 (steps step0 .. step0+nsteps, sources as in orc_rk4; y0 is not modified) and its
 * gradient with respect to every edge damping sigma_a[e] (grad laid out like sig; edges
 * with sigma_a[e] = 0 get 0: the supports of Phi/Psi are held fixed).  Every forward
 * state is kept (small problems only).  Per step m, backwards: add the residual of step m
 * to dJ/dU_m, run the reverse of the stage graph (as in orc_adjoint) and add
 * sum_i kbar_i^T (dA/dsigma) Y_i, with Y_i the stage inputs of the step from y_{m-1}.
 * Returns 0, or -1 when scratch cannot be allocated.
 */
int orc_misfit_grad_sigma(int ndim, const int64_t *T, double h, const double *sig, const double *y0,
                          int64_t nsteps, double dt, int64_t step0, int src_ns, const int64_t *src_idx,
                          const double *src_amp, double f_peak, double t_delay, int nr,
                          const int64_t *rec_idx, const double *target, double *J, double *grad)
{
    orc_grid g;
    orc_src s;
    int64_t n, len, k, j, m, tot, off;
    double *states, *k1, *k2, *k3, *Y2, *Y3, *Y4, *kb1, *kb2, *kb3, *kb4, *Yb, *yb, *yb_out, *res;
    int a, r;
    grid_from_args(&g, ndim, T, h, sig);
    s.ns = src_ns; s.idx = src_idx; s.amp = src_amp; s.f_peak = f_peak; s.t_delay = t_delay;
    n = grid_n(&g);
    len = (2 + 2 * (int64_t)ndim) * n;
    states = (double *)malloc(sizeof(double) * (size_t)(len * (nsteps + 1)));
    res = (double *)malloc(sizeof(double) * (size_t)(nsteps * (nr > 0 ? nr : 1)));
    k1 = (double *)malloc(sizeof(double) * (size_t)len);
    k2 = (double *)malloc(sizeof(double) * (size_t)len);
    k3 = (double *)malloc(sizeof(double) * (size_t)len);
    Y2 = (double *)malloc(sizeof(double) * (size_t)len);
    Y3 = (double *)malloc(sizeof(double) * (size_t)len);
    Y4 = (double *)malloc(sizeof(double) * (size_t)len);
    kb1 = (double *)malloc(sizeof(double) * (size_t)len);
    kb2 = (double *)malloc(sizeof(double) * (size_t)len);
    kb3 = (double *)malloc(sizeof(double) * (size_t)len);
    kb4 = (double *)malloc(sizeof(double) * (size_t)len);
    Yb = (double *)malloc(sizeof(double) * (size_t)len);
    yb = (double *)malloc(sizeof(double) * (size_t)len);
    yb_out = (double *)malloc(sizeof(double) * (size_t)len);
    if (!states || !res || !k1 || !k2 || !k3 || !Y2 || !Y3 || !Y4 || !kb1 || !kb2 || !kb3 || !kb4 || !Yb ||
        !yb || !yb_out) {
        free(states); free(res); free(k1); free(k2); free(k3); free(Y2); free(Y3); free(Y4);
        free(kb1); free(kb2); free(kb3); free(kb4); free(Yb); free(yb); free(yb_out);
        return -1;
    }
    /* forward run, every state kept; residuals of the receivers */
    memcpy(states, y0, sizeof(double) * (size_t)len);
    *J = 0.0;
    for (m = 1; m <= nsteps; m++) {
        double *y = states + m * len;
        memcpy(y, states + (m - 1) * len, sizeof(double) * (size_t)len);
        if (orc_rk4(ndim, T, h, sig, y, 1, dt, step0 + m - 1, src_ns, src_idx, src_amp, f_peak, t_delay, 0,
                    NULL, NULL) != 0)
            return -1;
        for (r = 0; r < nr; r++) {
            const double d = y[rec_idx[r]] - target[(m - 1) * nr + r];
            res[(m - 1) * nr + r] = d;
            *J += 0.5 * d * d;
        }
    }
    tot = 0;
    for (a = 0; a < ndim; a++) tot += g.T[a];
    for (j = 0; j < tot; j++) grad[j] = 0.0;
    for (j = 0; j < len; j++) yb[j] = 0.0;
    /* backwards */
    for (m = nsteps; m >= 1; m--) {
        const double *y = states + (m - 1) * len;
        const double t = (double)(step0 + m - 1) * dt;
        const orc_src *sp = src_ns > 0 ? &s : NULL;
        for (r = 0; r < nr; r++) yb[rec_idx[r]] += res[(m - 1) * nr + r];
        /* forward stage inputs of the step m-1 -> m */
        rhs(&g, y, k1, sp, t);
        for (j = 0; j < len; j++) Y2[j] = y[j] + 0.5 * dt * k1[j];
        rhs(&g, Y2, k2, sp, t + 0.5 * dt);
        for (j = 0; j < len; j++) Y3[j] = y[j] + 0.5 * dt * k2[j];
        rhs(&g, Y3, k3, sp, t + 0.5 * dt);
        for (j = 0; j < len; j++) Y4[j] = y[j] + dt * k3[j];
        /* reverse of the stage graph */
        for (j = 0; j < len; j++) {
            kb1[j] = dt / 6.0 * yb[j];
            kb2[j] = dt / 3.0 * yb[j];
            kb3[j] = dt / 3.0 * yb[j];
            kb4[j] = dt / 6.0 * yb[j];
            yb_out[j] = yb[j];
        }
        rhs_transpose(&g, kb4, Yb);
        for (j = 0; j < len; j++) { yb_out[j] += Yb[j]; kb3[j] += dt * Yb[j]; }
        rhs_transpose(&g, kb3, Yb);
        for (j = 0; j < len; j++) { yb_out[j] += Yb[j]; kb2[j] += 0.5 * dt * Yb[j]; }
        rhs_transpose(&g, kb2, Yb);
        for (j = 0; j < len; j++) { yb_out[j] += Yb[j]; kb1[j] += 0.5 * dt * Yb[j]; }
        rhs_transpose(&g, kb1, Yb);
        for (j = 0; j < len; j++) yb_out[j] += Yb[j];
        /* dJ/dsigma += sum_i kbar_i^T (dA/dsigma) Y_i */
        off = 0;
        for (a = 0; a < ndim; a++) {
            int64_t e;
            for (e = 0; e < g.T[a]; e++) {
                if (g.sig[a][e] == 0.0) continue;
                grad[off + e] += dA_contract(&g, a, e, kb1, y) + dA_contract(&g, a, e, kb2, Y2) +
                                 dA_contract(&g, a, e, kb3, Y3) + dA_contract(&g, a, e, kb4, Y4);
            }
            off += g.T[a];
        }
        memcpy(yb, yb_out, sizeof(double) * (size_t)len);
    }
    free(states); free(res); free(k1); free(k2); free(k3); free(Y2); free(Y3); free(Y4);
    free(kb1); free(kb2); free(kb3); free(kb4); free(Yb); free(yb); free(yb_out);
    (void)k;
    return 0;
}
