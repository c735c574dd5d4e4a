/*
 * fla_oracle.c -- plain, slow FP64 CPU oracle for the FLA hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark load this file's library.  The CUDA
 * library shares no code, header, table or helper with it.
 *
 * What it computes (Stafford & Rybdylova, "Interphase coupling for
 * gas-droplet flows using the fully Lagrangian approach"; equation numbers are
 * those of the paper, Sec. 2-3 and Appendices A-B):
 *
 *   carrier      analytic u(x,t) and grad u sampled on the mesh nodes and
 *                interpolated bi/trilinearly at the droplet (Eq. 3 needs
 *                u(x_d,t), Eq. 8 needs grad u(x_d,t); Sec. 4 interpolates
 *                them off the Eulerian mesh).
 *   advance      classical RK4 of  x' = v,  v' = (u - v)/St      (Eq. 3, Stokes drag)
 *                and  J' = W,  W' = (grad u . J - W)/St          (Eq. 8, Jacobian)
 *                with J(t0) = I, W(t0) = dv0/dx0, the d^2-law radius
 *                r^2 = r0^2 + delta (t - t0) in closed form (Eq. 4) and
 *                St = St0 (r/r0)^2 (Eq. 5).
 *   accumulate   per step the mass rate mdot and F + mdot v at the step's
 *                first RK stage, summed over the steps of a window (App. B,
 *                parcel level items a-b; F = m x'' is defined under Eq. 9).
 *   records      n = n0/|det J| (Eq. 6), h = h0 |det J| (Eq. 15) or the
 *                anisotropic precision matrix, a = n * acc / T_window.
 *   NW deposit   S = - sum_i K_i(x_c) a_i / sum_i K_i(x_c) at cell centres
 *                (Eqs. 13 and 16 with the signs of Eq. 9), Gaussian kernel of Eq. 14.
 *   PSI-CELL     S = -(1/V) sum_{i in cell} w_i a_i (Eqs. 10-11, box count).
 *
 * Each function loops over droplets and cells in ascending index order in
 * double precision.  Readings where the paper is silent are listed beside the
 * code that applies them.  Compile with -ffp-contract=off so that every
 * a*b+c rounds twice, as written.
 *
 * Threads: where droplets (one step of the advance) or cells (a deposit) are
 * independent, OpenMP spreads them over the host cores when the file is built
 * with -fopenmp.  Each droplet and each cell is still computed by the same
 * sequential code, so the results do not depend on the thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORA_PI 3.14159265358979323846
#define ORA_NO_DEADLINE 2147483647

enum { ORA_UNIFORM = 0, ORA_LINEAR = 1, ORA_TG2 = 2, ORA_JETVORT2 = 3, ORA_ABCJET3 = 4 };
enum { ORA_PENDING = 0, ORA_ACTIVE = 1, ORA_DEAD = 2 };

typedef struct {
    int kind, dim;
    double U[3];
    double A[9];          /* row-major, u_i += A_ij (x_j - xref_j) */
    double xref[3];
    int n_vort;
    double vort[16 * 5];  /* x0, yc, Gamma, rc, Uadv */
    double jet_width;
    double abc[3];
    double jet_amp, jet_radius;
} ora_carrier;

/* ------------------------------------------------------------------------ */
/* Carrier: analytic velocity and gradient G_ij = du_i/dx_j                  */
/* ------------------------------------------------------------------------ */

/* Lamb-Oseen vortex of circulation Gam and core radius rc centred at (xc,yc):
 * u_theta = Gam/(2 pi rho) (1 - exp(-rho^2/rc^2)).  Written as
 * u = f(s) (-dy, dx) with s = rho^2, f(s) = Gam/(2 pi) (1 - e^{-s/a})/s, a = rc^2. */
static void lamb_oseen(double Gam, double rc, double xc, double yc, const double* x,
                       double* u, double* G)
{
    double dx = x[0] - xc, dy = x[1] - yc;
    double s = dx * dx + dy * dy;
    double a = rc * rc;
    double c = Gam / (2.0 * ORA_PI);
    double X = s / a;
    double h, g;   /* f = (c/a) h(X),  f'(s) = (c/a^2) g(X) */
    if (X < 1e-3) {
        /* Taylor series of h = (1 - e^{-X})/X and g = (X e^{-X} - (1 - e^{-X}))/X^2 */
        h = 1.0 - X / 2.0 + X * X / 6.0 - X * X * X / 24.0;
        g = -0.5 + X / 3.0 - X * X / 8.0 + X * X * X / 30.0;
    } else {
        double em = expm1(-X);        /* e^{-X} - 1 */
        h = -em / X;
        g = (X * exp(-X) + em) / (X * X);
    }
    double f = (c / a) * h;
    double fp = (c / (a * a)) * g;
    u[0] += -dy * f;
    u[1] += dx * f;
    G[0] += -dy * fp * 2.0 * dx;          /* d(-dy f)/dx */
    G[1] += -f - dy * fp * 2.0 * dy;      /* d(-dy f)/dy */
    G[2] += f + dx * fp * 2.0 * dx;       /* d(dx f)/dx  */
    G[3] += dx * fp * 2.0 * dy;           /* d(dx f)/dy  */
}

void ora_carrier_eval(const ora_carrier* c, double t, const double* x, double* u, double* G)
{
    int d = c->dim;
    for (int i = 0; i < d; ++i) u[i] = 0.0;
    for (int i = 0; i < d * d; ++i) G[i] = 0.0;
    switch (c->kind) {
    case ORA_UNIFORM:
        for (int i = 0; i < d; ++i) u[i] = c->U[i];
        break;
    case ORA_LINEAR:
        for (int i = 0; i < d; ++i) {
            u[i] = c->U[i];
            for (int j = 0; j < d; ++j) {
                u[i] += c->A[i * 3 + j] * (x[j] - c->xref[j]);
                G[i * d + j] = c->A[i * 3 + j];
            }
        }
        break;
    case ORA_TG2: {
        double sx = sin(ORA_PI * x[0]), cx = cos(ORA_PI * x[0]);
        double sy = sin(ORA_PI * x[1]), cy = cos(ORA_PI * x[1]);
        u[0] = sx * cy;
        u[1] = -cx * sy;
        G[0] = ORA_PI * cx * cy;
        G[1] = -ORA_PI * sx * sy;
        G[2] = ORA_PI * sx * sy;
        G[3] = -ORA_PI * cx * cy;
        break;
    }
    case ORA_JETVORT2: {
        double w = c->jet_width;
        double eta = (x[1] - 0.5) / w;
        double uj = exp(-eta * eta);
        u[0] = uj;
        G[1] = -2.0 * eta / w * uj;
        for (int k = 0; k < c->n_vort; ++k) {
            const double* v = c->vort + 5 * k;
            double xc = v[0] + v[4] * t;
            xc = xc - floor(xc);                      /* wrapped into [0,1) */
            for (int img = -1; img <= 1; ++img)       /* periodic images in x */
                lamb_oseen(v[2], v[3], xc + img, v[1], x, u, G);
        }
        break;
    }
    case ORA_ABCJET3: {
        double A = c->abc[0], B = c->abc[1], C = c->abc[2];
        double k = 2.0 * ORA_PI;
        double sxv = sin(k * x[0]), cxv = cos(k * x[0]);
        double syv = sin(k * x[1]), cyv = cos(k * x[1]);
        double szv = sin(k * x[2]), czv = cos(k * x[2]);
        u[0] = A * szv + C * cyv;
        u[1] = B * sxv + A * czv;
        u[2] = C * syv + B * cxv;
        G[0 * 3 + 1] = -k * C * syv;
        G[0 * 3 + 2] = k * A * czv;
        G[1 * 3 + 0] = k * B * cxv;
        G[1 * 3 + 2] = -k * A * szv;
        G[2 * 3 + 0] = -k * B * sxv;
        G[2 * 3 + 1] = k * C * cyv;
        double rx = x[0] - 0.5, ry = x[1] - 0.5, r2j = c->jet_radius * c->jet_radius;
        double e = c->jet_amp * exp(-(rx * rx + ry * ry) / r2j);
        u[2] += e;
        G[2 * 3 + 0] += -2.0 * rx / r2j * e;
        G[2 * 3 + 1] += -2.0 * ry / r2j * e;
        break;
    }
    default:
        break;
    }
}

/* Node values for carrier time t.  Nodes at i/N along each axis, linear index
 * with x fastest; each node holds u (dim) then G (dim*dim, row-major). */
void ora_carrier_nodes(const ora_carrier* c, double t, int N, double* nodes)
{
    int d = c->dim, nn = N + 1, stride = d + d * d;
    long total = (d == 2) ? (long)nn * nn : (long)nn * nn * nn;
#pragma omp parallel for schedule(static)
    for (long k = 0; k < total; ++k) {
        double x[3];
        long r = k;
        for (int a = 0; a < d; ++a) { x[a] = (double)(r % nn) / N; r /= nn; }
        ora_carrier_eval(c, t, x, nodes + k * stride, nodes + k * stride + d);
    }
}

/* Bi/trilinear interpolation of the node values at x.  The containing cell
 * index is clamped to [0, N-1], so positions just outside the domain (RK
 * stages) are extrapolated from the edge cell. */
void ora_interp(const double* nodes, int d, int N, const double* x, double* u, double* G)
{
    int nn = N + 1, stride = d + d * d;
    int ic[3];
    double f[3];
    for (int a = 0; a < d; ++a) {
        double s = x[a] * N;
        int i = (int)floor(s);
        if (i < 0) i = 0;
        if (i > N - 1) i = N - 1;
        ic[a] = i;
        f[a] = s - i;
    }
    for (int q = 0; q < stride; ++q) {
        double acc = 0.0;
        int ncorner = 1 << d;
        for (int cnr = 0; cnr < ncorner; ++cnr) {
            double w = 1.0;
            long idx = 0, mul = 1;
            for (int a = 0; a < d; ++a) {
                int bit = (cnr >> a) & 1;
                w *= bit ? f[a] : (1.0 - f[a]);
                idx += (long)(ic[a] + bit) * mul;
                mul *= nn;
            }
            acc += w * nodes[idx * stride + q];
        }
        if (q < d) u[q] = acc; else G[q - d] = acc;
    }
}

/* ------------------------------------------------------------------------ */
/* Advance                                                                   */
/* ------------------------------------------------------------------------ */

typedef struct {
    int dim, N;
    int cloud;            /* 0: FLA (x, v, J, W), 1: plain LPT (x, v) */
    double dt, delta;     /* step, d^2-law rate; r0 = 1 */
    const ora_carrier* car;
    int use_mesh;         /* 1: sample nodes and interpolate; 0: analytic carrier at x */
    int carrier_period;   /* steps per carrier re-sample, 0 = steady */
    int n_batches;
    const int* step_start;
    const int* step_dead;
    const double* St0;
    const double* given_nodes;   /* non-NULL: these node values ((N+1)^d x (d + d*d)) instead of the
                                    analytic carrier, e.g. a Navier-Stokes carrier's (two-way coupling) */
} ora_setup;

/* Steps at which a release stops: first step s >= s0 at which the closed-form
 * r^2 = 1 + delta (s - s0) dt falls below max(0.01, 4 dt / St0).  Beyond it St
 * is too small for an explicit step and the droplet has nearly vanished
 * (r^2 -> 0 makes Eq. 3 singular; the paper does not reach that point). */
int ora_step_dead(double St0, double delta, double dt, int step_start)
{
    if (!(delta < 0.0)) return ORA_NO_DEADLINE;
    double thr = 0.01;
    if (4.0 * dt / St0 > thr) thr = 4.0 * dt / St0;
    double est = (1.0 - thr) / (-delta) / dt;      /* steps until threshold */
    if (est > 2.0e9) return ORA_NO_DEADLINE;
    long s = (long)step_start + (long)floor(est) - 2;
    if (s < step_start) s = step_start;
    while (!(1.0 + delta * (double)(s - step_start) * dt < thr)) ++s;
    if (s > 2147483646L) return ORA_NO_DEADLINE;
    return (int)s;
}

typedef struct {
    const ora_setup* S;
    const double* nodes;  /* NULL: analytic */
    double tc;            /* carrier time of the current frozen carrier step */
} ora_flow;

static void flow_at(const ora_flow* F, const double* x, double* u, double* G)
{
    if (F->nodes) ora_interp(F->nodes, F->S->dim, F->S->N, x, u, G);
    else ora_carrier_eval(F->S->car, F->tc, x, u, G);
}

/* Right-hand side of the droplet system at time t for state y.
 * FLA: y = (x[d], v[d], J[d*d], W[d*d]);  LPT: y = (x[d], v[d]). */
static void rhs(const ora_flow* F, double St, const double* y, double* f)
{
    const ora_setup* S = F->S;
    int d = S->dim;
    double u[3], G[9];
    flow_at(F, y, u, G);
    const double* v = y + d;
    for (int a = 0; a < d; ++a) {
        f[a] = v[a];                                  /* x' = v            */
        f[d + a] = (u[a] - v[a]) / St;                /* v' = (u - v)/St   (Eq. 3) */
    }
    if (S->cloud == 0) {
        const double* J = y + 2 * d;
        const double* W = y + 2 * d + d * d;
        for (int i = 0; i < d; ++i)
            for (int k = 0; k < d; ++k) {
                double GJ = 0.0;                      /* (grad u . J)_ik = sum_j G_ij J_jk */
                for (int j = 0; j < d; ++j) GJ += G[i * d + j] * J[j * d + k];
                f[2 * d + i * d + k] = W[i * d + k];                     /* J' = W */
                f[2 * d + d * d + i * d + k] = (GJ - W[i * d + k]) / St; /* W' = (G J - W)/St (Eq. 8) */
            }
    }
}

/* r^2/r0^2 from the closed-form integral of Eq. 4 with r0 = 1. */
static double r2_at(double delta, double t, double t0) { return 1.0 + delta * (t - t0); }

/* Advance steps [step0, step0 + nsteps).  y: n x ny doubles, acc: n x (1+d),
 * status per droplet (pending / active / dead), batch per droplet.
 * reset_acc zeroes the window sums first.  Returns 0. */
int ora_advance(const ora_setup* S, int step0, int nsteps, int n, double* y, double* acc,
                int* status, const int* batch, int reset_acc)
{
    int d = S->dim;
    int ny = (S->cloud == 0) ? 2 * d + 2 * d * d : 2 * d;
    int na = 1 + d;
    int nn = S->N + 1;
    long nnodes = (d == 2) ? (long)nn * nn : (long)nn * nn * nn;
    double* nodes = NULL;
    double nodes_t = -1.0;
    if (S->use_mesh) nodes = (double*)malloc(sizeof(double) * nnodes * (d + d * d));

    if (reset_acc)
        for (long i = 0; i < (long)n * na; ++i) acc[i] = 0.0;

    for (int s = step0; s < step0 + nsteps; ++s) {
        double t = s * S->dt;
        ora_flow F = { S, NULL, 0.0 };
        /* carrier frozen over each carrier step, sampled at its start (reading: the
         * paper's carrier is a CFD solution updated once per carrier time step) */
        F.tc = (S->carrier_period > 0) ? (double)((s / S->carrier_period) * S->carrier_period) * S->dt : 0.0;
        if (S->given_nodes) {
            F.nodes = S->given_nodes;
        } else if (S->use_mesh) {
            if (F.tc != nodes_t) { ora_carrier_nodes(S->car, F.tc, S->N, nodes); nodes_t = F.tc; }
            F.nodes = nodes;
        }
#pragma omp parallel for schedule(dynamic, 256)
        for (int i = 0; i < n; ++i) {
            double k1[24], k2[24], k3[24], k4[24], ys[24];   /* ny <= 24 */
            int b = batch[i];
            double* yi = y + (long)i * ny;
            double* ai = acc + (long)i * na;
            if (status[i] == ORA_PENDING && s == S->step_start[b]) {
                /* release: v0 = u(x0), J = I, W = dv0/dx0 = grad u(x0) (Eq. 8 initial data) */
                double u[3], G[9];
                flow_at(&F, yi, u, G);
                for (int a = 0; a < d; ++a) yi[d + a] = u[a];
                if (S->cloud == 0)
                    for (int q = 0; q < d * d; ++q) {
                        yi[2 * d + q] = (q % (d + 1) == 0) ? 1.0 : 0.0;
                        yi[2 * d + d * d + q] = G[q];
                    }
                for (int a = 0; a < na; ++a) ai[a] = 0.0;
                status[i] = ORA_ACTIVE;
            }
            if (status[i] != ORA_ACTIVE) continue;
            if (s >= S->step_dead[b]) { status[i] = ORA_DEAD; continue; }

            double t0 = S->step_start[b] * S->dt;
            double St0 = S->St0[b];
            double h = S->dt;
            double St_a = St0 * r2_at(S->delta, t, t0);
            double St_b = St0 * r2_at(S->delta, t + 0.5 * h, t0);
            double St_c = St0 * r2_at(S->delta, t + h, t0);

            /* window sums at the first stage (left rectangle rule over the substeps,
             * App. B items a-b): mdot = d(r^3)/dt = 1.5 delta r, F = m (u - v)/St */
            {
                double u[3], G[9];
                flow_at(&F, yi, u, G);
                double r2 = r2_at(S->delta, t, t0);
                double r = sqrt(r2);
                double m = r2 * r;
                double mdot = 1.5 * S->delta * r;
                ai[0] += h * mdot;
                for (int a = 0; a < d; ++a) {
                    double Fa = m * (u[a] - yi[d + a]) / St_a;
                    ai[1 + a] += h * (Fa + mdot * yi[d + a]);
                }
            }
            /* classical RK4 */
            rhs(&F, St_a, yi, k1);
            for (int q = 0; q < ny; ++q) ys[q] = yi[q] + 0.5 * h * k1[q];
            rhs(&F, St_b, ys, k2);
            for (int q = 0; q < ny; ++q) ys[q] = yi[q] + 0.5 * h * k2[q];
            rhs(&F, St_b, ys, k3);
            for (int q = 0; q < ny; ++q) ys[q] = yi[q] + h * k3[q];
            rhs(&F, St_c, ys, k4);
            for (int q = 0; q < ny; ++q)
                yi[q] = yi[q] + h / 6.0 * (k1[q] + 2.0 * k2[q] + 2.0 * k3[q] + k4[q]);
            /* leaving [0,1]^d ends the trajectory (reading: the synthetic domain has
             * outflow boundaries; its window sums are dropped) */
            for (int a = 0; a < d; ++a)
                if (yi[a] < 0.0 || yi[a] > 1.0) status[i] = ORA_DEAD;
        }
    }
    free(nodes);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Cell keys (mesh binning used by PSI-CELL and the cell list)               */
/* ------------------------------------------------------------------------ */

/* key = linear index of the containing cell, x fastest; floor(x N) clamped to
 * N-1 so that x = 1 belongs to the last cell; 0xFFFFFFFF for droplets that are
 * not active or lie outside [0,1]^d.  With fp32 set the product x*N is formed
 * in single precision, as a single-precision kernel forms it. */
void ora_cell_keys(int d, int N, int n, const double* x, const int* status, int fp32, uint32_t* keys)
{
    for (int i = 0; i < n; ++i) {
        const double* xi = x + (long)i * d;
        uint32_t key = 0, mul = 1;
        int ok = (status[i] == ORA_ACTIVE);
        for (int a = 0; a < d && ok; ++a) {
            if (!(xi[a] >= 0.0 && xi[a] <= 1.0)) { ok = 0; break; }
            double s = fp32 ? (double)((float)xi[a] * (float)N) : xi[a] * N;
            long c = (long)floor(s);
            if (c > N - 1) c = N - 1;
            key += (uint32_t)c * mul;
            mul *= (uint32_t)N;
        }
        keys[i] = ok ? key : 0xFFFFFFFFu;
    }
}

/* ------------------------------------------------------------------------ */
/* Records and the Nadaraya-Watson deposit                                   */
/* ------------------------------------------------------------------------ */

typedef struct {
    int dim, N;
    int kernel;          /* 0: spherical kernel of Eq. 14 with h of Eq. 15; 1: J-scaled anisotropic */
    double h_min, h_max; /* clamps of the smoothing length (reading: paper gives none) */
    double p;            /* h = h0 |det J|^p; p = 1 is Eq. 15 */
    double window_dt;    /* length of the window the sums cover */
    int per_cell;        /* 1: multiply S by the cell volume (per-cell amounts) */
    int fp32_decision;   /* 1: the q <= 9 truncation is decided on single-precision operands */
    int plain;           /* with fp32_decision: det J decided in single precision throughout */
    const int* fold;     /* per droplet, or NULL: 1 = J is the fold guard's double-precision copy */
    const float* mlp;    /* learned bandwidth correction, or NULL */
} ora_dep;

/* learned bandwidth correction, defined at the end of this file */
void ora_mlp_features(int d, const double* J, double n0, double h0, double dx, double* f);
double ora_mlp_forward(const float* P, const double* f, const double* fe, double* bound, double* act, double* zs);
void ora_mlp_backward(const float* P, const double* f, double dLdc, double* grad);

typedef struct {
    double x[3];
    double n;            /* n0/|det J| */
    double detJ;
    double a[4];         /* n * acc / T_window */
    double h;            /* isotropic smoothing length */
    double P[9];         /* anisotropic precision matrix Sigma^{-1} */
    double pref;         /* kernel prefactor: 1/h (Eq. 14) or det(Sigma)^{-1/2} */
    float xf[3];         /* single-precision operands of the truncation decision */
    float r2max_f;
    float Pf[9];
    double c;            /* learned correction g(f) (0 without the network) */
    int dh_dc;           /* 1 when the bandwidth moves with c: c inside (-2, 2), away from folds, h not
                            clamped (spherical) or the trace cap inactive (J-scaled) */
    double f[6];         /* the network's features */
} ora_rec;

static double det_d(int d, const double* J)
{
    if (d == 2) return J[0] * J[3] - J[1] * J[2];
    return J[0] * (J[4] * J[8] - J[5] * J[7])
         - J[1] * (J[3] * J[8] - J[5] * J[6])
         + J[2] * (J[3] * J[7] - J[4] * J[6]);
}

/* inverse of a symmetric d x d matrix by the adjugate */
static void inv_sym(int d, const double* S, double det, double* P)
{
    if (d == 2) {
        P[0] = S[3] / det; P[3] = S[0] / det;
        P[1] = -S[1] / det; P[2] = P[1];
        return;
    }
    double c00 = S[4] * S[8] - S[5] * S[7];
    double c01 = S[5] * S[6] - S[3] * S[8];
    double c02 = S[3] * S[7] - S[4] * S[6];
    double c11 = S[0] * S[8] - S[2] * S[6];
    double c12 = S[2] * S[3] - S[0] * S[5];
    double c22 = S[0] * S[4] - S[1] * S[3];
    P[0] = c00 / det; P[1] = c01 / det; P[2] = c02 / det;
    P[3] = P[1];      P[4] = c11 / det; P[5] = c12 / det;
    P[6] = P[2];      P[7] = P[5];      P[8] = c22 / det;
}

/* Single-precision operands of the truncation decision, formed as a
 * single-precision kernel forms them (reading: a floating-point comparison
 * that decides an integer is taken in the kernel's precision on both sides).
 *  - |det J|: in double from the single-precision entries (2D, products exact);
 *    in 3D the cofactor expansion in single precision unless |det| < 1e-2 times
 *    the product of the rows' L1 norms (near a fold), then in double; in double
 *    from the given J for a droplet in the fold guard; and in single precision
 *    throughout in the plain mode;
 *  - spherical kernel: h = clamp(h0 |det J|^p, h_min, h_max) in double, rounded,
 *    and r2max = 9 h^2 formed in double from the rounded h and rounded;
 *  - J-scaled kernel: Sigma and its inverse in single precision, one rounding
 *    per operation, in the order written below. */
static double det_decision(int d, const double* J, int plain, int fold)
{
    float j[9];
    for (int q = 0; q < d * d; ++q) j[q] = (float)J[q];
    if (plain) {
        /* plain single precision: the cofactor expansion in float */
        if (d == 2) return (double)(j[0] * j[3] - j[1] * j[2]);
        return (double)(j[0] * (j[4] * j[8] - j[5] * j[7]) - j[1] * (j[3] * j[8] - j[5] * j[6])
                        + j[2] * (j[3] * j[7] - j[4] * j[6]));
    }
    /* a droplet in the fold guard: det J in double from its double-precision J */
    if (fold || d == 2) return det_d(d, J);
    float detf = j[0] * (j[4] * j[8] - j[5] * j[7]) - j[1] * (j[3] * j[8] - j[5] * j[6])
               + j[2] * (j[3] * j[7] - j[4] * j[6]);
    float H = (fabsf(j[0]) + fabsf(j[1]) + fabsf(j[2])) * (fabsf(j[3]) + fabsf(j[4]) + fabsf(j[5]))
            * (fabsf(j[6]) + fabsf(j[7]) + fabsf(j[8]));
    if (fabsf(detf) < 0.01f * H) return det_d(3, J);
    return (double)detf;
}

static void aniso_decision(const ora_dep* D, const double* J, double h0, float* Pf)
{
    int d = D->dim;
    float j[9], S[9];
    for (int q = 0; q < d * d; ++q) j[q] = (float)J[q];
    float h02 = (float)h0 * (float)h0;
    float room = (float)(D->h_max * D->h_max - d * D->h_min * D->h_min);
    float hmin2 = (float)(D->h_min * D->h_min);
    float tr0 = 0.0f;
    for (int i = 0; i < d; ++i)
        for (int k = 0; k < d; ++k) {
            float sum = 0.0f;
            for (int q = 0; q < d; ++q) sum = sum + j[i * d + q] * j[k * d + q];
            S[i * d + k] = h02 * sum;
            if (i == k) tr0 = tr0 + S[i * d + k];
        }
    if (tr0 > room) {
        float f = room / tr0;
        for (int q = 0; q < d * d; ++q) S[q] = S[q] * f;
    }
    for (int i = 0; i < d; ++i) S[i * d + i] = S[i * d + i] + hmin2;
    if (d == 2) {
        float dS = S[0] * S[3] - S[1] * S[2];
        float inv = 1.0f / dS;
        Pf[0] = S[3] * inv; Pf[3] = S[0] * inv; Pf[1] = -S[1] * inv; Pf[2] = Pf[1];
        return;
    }
    float c00 = S[4] * S[8] - S[5] * S[7];
    float c01 = S[5] * S[6] - S[3] * S[8];
    float c02 = S[3] * S[7] - S[4] * S[6];
    float c11 = S[0] * S[8] - S[2] * S[6];
    float c12 = S[2] * S[3] - S[0] * S[5];
    float c22 = S[0] * S[4] - S[1] * S[3];
    float dS = S[0] * c00 + S[1] * c01 + S[2] * c02;
    float inv = 1.0f / dS;
    Pf[0] = c00 * inv; Pf[1] = c01 * inv; Pf[2] = c02 * inv;
    Pf[3] = Pf[1];     Pf[4] = c11 * inv; Pf[5] = c12 * inv;
    Pf[6] = Pf[2];     Pf[7] = Pf[5];     Pf[8] = c22 * inv;
}

/* Record of one active droplet: Eq. 6 number density, Eq. 15 smoothing length
 * or the J-scaled covariance Sigma = f h0^2 J J^T + h_min^2 I (reading: the
 * push-forward of the spherical kernel by J, kept positive definite at folds by
 * the h_min^2 I floor), where f = min(1, (h_max^2 - d h_min^2)/tr(h0^2 J J^T))
 * caps tr(Sigma) <= h_max^2 so that the support stays within 3 h_max. */
void ora_record(const ora_dep* D, const double* x, const double* J, const double* acc,
                double n0, double h0, int fold, ora_rec* r)
{
    int d = D->dim;
    memset(r, 0, sizeof(*r));
    for (int a = 0; a < d; ++a) { r->x[a] = x[a]; r->xf[a] = (float)x[a]; }
    double det = det_d(d, J);
    double adet = fabs(det);
    r->detJ = det;
    r->n = n0 / (adet > 1e-12 ? adet : 1e-12);            /* Eq. 6, floored at folds */
    for (int a = 0; a < 1 + d; ++a) r->a[a] = r->n * acc[a] / D->window_dt;
    if (D->kernel == 0) {
        double h = (D->p == 1.0) ? h0 * adet : h0 * pow(adet, D->p);   /* Eq. 15 */
        double corr = 1.0;
        if (D->mlp) {      /* learned correction: h <- h exp(clip(g(f), -2, 2)) */
            ora_mlp_features(d, J, n0, h0, 1.0 / D->N, r->f);
            r->c = ora_mlp_forward(D->mlp, r->f, NULL, NULL, NULL, NULL);
            /* it stays off near fold caustics (|det J| < 1e-2, in the precision of the
             * truncation decision), where the plain kernel is the fallback: n is
             * singular there and a bandwidth learned away from folds does not transfer */
            double ad_fold = D->fp32_decision ? fabs(det_decision(d, J, D->plain, fold)) : adet;
            if (ad_fold >= 1e-2) {
                double ct = r->c < -2.0 ? -2.0 : (r->c > 2.0 ? 2.0 : r->c);
                corr = exp(ct);
                h *= corr;
                r->dh_dc = (r->c > -2.0 && r->c < 2.0 && h > D->h_min && h < D->h_max);
            }
        }
        if (h < D->h_min) h = D->h_min;
        if (h > D->h_max) h = D->h_max;
        r->h = h;
        r->pref = 1.0 / h;                                 /* Eq. 14 prefactor */
        double ad = fabs(det_decision(d, J, D->plain, fold));
        double hd = (D->p == 1.0) ? h0 * ad : h0 * pow(ad, D->p);
        hd *= corr;
        if (hd < D->h_min) hd = D->h_min;
        if (hd > D->h_max) hd = D->h_max;
        r->r2max_f = (float)(9.0 * (double)(float)hd * (double)(float)hd);
    } else {
        /* learned correction: the Lagrangian bandwidth h0 of the J-scaled kernel
         * becomes h0 exp(clip(g(f), -2, 2)), off near folds as above */
        double h0s = h0;
        int moves = 0;
        if (D->mlp) {
            ora_mlp_features(d, J, n0, h0, 1.0 / D->N, r->f);
            r->c = ora_mlp_forward(D->mlp, r->f, NULL, NULL, NULL, NULL);
            double ad_fold = D->fp32_decision ? fabs(det_decision(d, J, D->plain, fold)) : adet;
            if (ad_fold >= 1e-2) {
                double ct = r->c < -2.0 ? -2.0 : (r->c > 2.0 ? 2.0 : r->c);
                h0s = h0 * exp(ct);
                moves = r->c > -2.0 && r->c < 2.0;
            }
        }
        double Sg[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        double tr0 = 0.0;
        for (int i = 0; i < d; ++i)
            for (int k = 0; k < d; ++k) {
                double s = 0.0;
                for (int j = 0; j < d; ++j) s += J[i * d + j] * J[k * d + j];
                Sg[i * d + k] = h0s * h0s * s;
                if (i == k) tr0 += Sg[i * d + k];
            }
        double room = D->h_max * D->h_max - d * D->h_min * D->h_min;
        /* Sigma moves with c only while the trace cap is inactive */
        r->dh_dc = moves && !(tr0 > room);
        if (tr0 > room) {
            double f = room / tr0;
            for (int q = 0; q < d * d; ++q) Sg[q] *= f;
        }
        for (int i = 0; i < d; ++i) Sg[i * d + i] += D->h_min * D->h_min;
        double tr = 0.0;
        for (int i = 0; i < d; ++i) tr += Sg[i * d + i];
        double dS = det_d(d, Sg);
        inv_sym(d, Sg, dS, r->P);
        r->pref = 1.0 / sqrt(dS);
        r->h = sqrt(tr);
        aniso_decision(D, J, h0s, r->Pf);
    }
}

/* Squared distance / Mahalanobis form and the q <= 9 (three sigma) truncation
 * of the Gaussian (reading: the paper's kernel has unbounded support). */
static int in_support(const ora_dep* D, const ora_rec* r, const double* xc, const float* xcf, double* q_out)
{
    int d = D->dim;
    double dv[3];
    for (int a = 0; a < d; ++a) dv[a] = xc[a] - r->x[a];
    double q;
    if (D->kernel == 0) {
        double r2 = 0.0;
        for (int a = 0; a < d; ++a) r2 += dv[a] * dv[a];
        q = r2 / (r->h * r->h);
    } else {
        q = 0.0;
        for (int i = 0; i < d; ++i)
            for (int k = 0; k < d; ++k) q += dv[i] * r->P[i * d + k] * dv[k];
    }
    *q_out = q;
    if (!D->fp32_decision) return q <= 9.0;
    /* the same decision on single-precision operands, in a fixed operation order:
     * differences, then products and sums, each rounded to single precision */
    float df[3] = {0.0f, 0.0f, 0.0f};
    for (int a = 0; a < d; ++a) df[a] = xcf[a] - r->xf[a];
    if (D->kernel == 0) {
        float r2 = df[0] * df[0];
        r2 = fmaf(df[1], df[1], r2);
        if (d == 3) r2 = fmaf(df[2], df[2], r2);
        return r2 <= r->r2max_f;
    } else {
        float pd[3] = {0.0f, 0.0f, 0.0f};
        for (int i = 0; i < d; ++i) {
            float s = r->Pf[i * d + 0] * df[0];
            for (int k = 1; k < d; ++k) s = fmaf(r->Pf[i * d + k], df[k], s);
            pd[i] = s;
        }
        float qf = pd[0] * df[0];
        for (int i = 1; i < d; ++i) qf = fmaf(pd[i], df[i], qf);
        return qf <= 9.0f;
    }
}

static double cell_volume(const ora_dep* D) { double h = 1.0 / D->N; return D->dim == 2 ? h * h : h * h * h; }

static void cell_centre(int d, int N, long c, double* xc, float* xcf)
{
    for (int a = 0; a < d; ++a) {
        long i = c % N; c /= N;
        xc[a] = (i + 0.5) / N;
        xcf[a] = (float)xc[a];
    }
}

/* A droplet contributes to a deposit when it is active and inside [0,1]^d. */
static int contributes(int d, const double* x, int status)
{
    if (status != ORA_ACTIVE) return 0;
    for (int a = 0; a < d; ++a) if (!(x[a] >= 0.0 && x[a] <= 1.0)) return 0;
    return 1;
}

/* Nadaraya-Watson source terms (Eqs. 13 and 16 with the signs of Eq. 9) at the
 * listed cells, brute force over all droplets in ascending index order:
 *   D_c = sum_i K_i(x_c),  S_mass = -sum_i K_i a_m,i / D_c,  S_mom = -sum_i K_i a_mom,i / D_c,
 * and S = 0 where D_c = 0.  cells == NULL means every cell in order.
 * Inputs per droplet: x (d), J (d*d), acc (1+d), status, batch; per batch n0, h0. */
int ora_nw_deposit(const ora_dep* D, int n, const double* x, const double* J, const double* acc,
                   const int* status, const int* batch, const double* n0, const double* h0,
                   long n_out, const long* cells, double* S_mass, double* S_mom, double* Dsum)
{
    int d = D->dim;
    ora_rec* rec = (ora_rec*)malloc(sizeof(ora_rec) * (n > 0 ? n : 1));
    int* use = (int*)malloc(sizeof(int) * (n > 0 ? n : 1));
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) {
        use[i] = contributes(d, x + (long)i * d, status[i]);
        if (use[i])
            ora_record(D, x + (long)i * d, J + (long)i * d * d, acc + (long)i * (1 + d),
                       n0[batch[i]], h0[batch[i]], D->fold ? D->fold[i] : 0, &rec[i]);
    }
    double V = cell_volume(D);
#pragma omp parallel for schedule(dynamic, 16)
    for (long o = 0; o < n_out; ++o) {
        long c = cells ? cells[o] : o;
        double xc[3]; float xcf[3];
        cell_centre(d, D->N, c, xc, xcf);
        double den = 0.0, num[4] = {0, 0, 0, 0};
        for (int i = 0; i < n; ++i) {
            if (!use[i]) continue;
            double q;
            if (!in_support(D, &rec[i], xc, xcf, &q)) continue;
            double w = rec[i].pref * exp(-0.5 * q);          /* Eq. 14 */
            den += w;
            for (int a = 0; a < 1 + d; ++a) num[a] += w * rec[i].a[a];
        }
        double scale = D->per_cell ? V : 1.0;
        S_mass[o] = den > 0.0 ? -num[0] / den * scale : 0.0;
        for (int a = 0; a < d; ++a) S_mom[o * d + a] = den > 0.0 ? -num[1 + a] / den * scale : 0.0;
        Dsum[o] = den;
    }
    free(rec); free(use);
    return 0;
}

static int cmp_int(const void* a, const void* b)
{
    int x = *(const int*)a, y = *(const int*)b;
    return (x > y) - (x < y);
}

/* The same deposit through a cell list: droplets are binned by cell key, each
 * cell collects the droplets of the cells within R = floor(3 h_max/dx + 1/2) + 1
 * cells (every droplet whose truncated kernel can reach the centre), sorts the
 * candidates by index and sums in that order.  Gives bit-identical results to
 * ora_nw_deposit. */
int ora_nw_deposit_celllist_cells(const ora_dep* D, int n, const double* x, const double* J, const double* acc,
                                  const int* status, const int* batch, const double* n0, const double* h0,
                                  long n_out, const long* cells, double* S_mass, double* S_mom, double* Dsum);

int ora_nw_deposit_celllist(const ora_dep* D, int n, const double* x, const double* J, const double* acc,
                            const int* status, const int* batch, const double* n0, const double* h0,
                            double* S_mass, double* S_mom, double* Dsum)
{
    int d = D->dim, N = D->N;
    long nc = (d == 2) ? (long)N * N : (long)N * N * N;
    return ora_nw_deposit_celllist_cells(D, n, x, J, acc, status, batch, n0, h0, nc, NULL, S_mass, S_mom, Dsum);
}

/* Cell-list deposit at the listed cells (NULL: every cell in order). */
int ora_nw_deposit_celllist_cells(const ora_dep* D, int n, const double* x, const double* J, const double* acc,
                                  const int* status, const int* batch, const double* n0, const double* h0,
                                  long n_out, const long* cells, double* S_mass, double* S_mom, double* Dsum)
{
    int d = D->dim, N = D->N;
    long nc = (d == 2) ? (long)N * N : (long)N * N * N;
    uint32_t* keys = (uint32_t*)malloc(sizeof(uint32_t) * (n > 0 ? n : 1));
    ora_cell_keys(d, N, n, x, status, 0, keys);
    long* start = (long*)calloc(nc + 1, sizeof(long));
    int* list = (int*)malloc(sizeof(int) * (n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) if (keys[i] != 0xFFFFFFFFu) start[keys[i] + 1]++;
    for (long c = 0; c < nc; ++c) start[c + 1] += start[c];
    long* fill = (long*)malloc(sizeof(long) * nc);
    memcpy(fill, start, sizeof(long) * nc);
    for (int i = 0; i < n; ++i) if (keys[i] != 0xFFFFFFFFu) list[fill[keys[i]]++] = i;
    ora_rec* rec = (ora_rec*)malloc(sizeof(ora_rec) * (n > 0 ? n : 1));
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i)
        if (keys[i] != 0xFFFFFFFFu)
            ora_record(D, x + (long)i * d, J + (long)i * d * d, acc + (long)i * (1 + d),
                       n0[batch[i]], h0[batch[i]], D->fold ? D->fold[i] : 0, &rec[i]);
    int R = (int)floor(3.0 * D->h_max * N + 0.5) + 1;
    double V = cell_volume(D);
#pragma omp parallel
    {
    int* cand = (int*)malloc(sizeof(int) * (n > 0 ? n : 1));   /* one candidate list per thread */
#pragma omp for schedule(dynamic, 16)
    for (long o = 0; o < n_out; ++o) {
        long c = cells ? cells[o] : o;
        int ci[3] = {0, 0, 0};
        long r = c;
        for (int a = 0; a < d; ++a) { ci[a] = (int)(r % N); r /= N; }
        int nca = 0;
        int lo[3], hi[3];
        for (int a = 0; a < 3; ++a) { lo[a] = 0; hi[a] = 0; }
        for (int a = 0; a < d; ++a) {
            lo[a] = ci[a] - R < 0 ? 0 : ci[a] - R;
            hi[a] = ci[a] + R > N - 1 ? N - 1 : ci[a] + R;
        }
        for (int kz = lo[2]; kz <= hi[2]; ++kz)
            for (int ky = lo[1]; ky <= hi[1]; ++ky)
                for (int kx = lo[0]; kx <= hi[0]; ++kx) {
                    long b = kx + (long)N * ky + (long)N * N * kz;
                    for (long m = start[b]; m < start[b + 1]; ++m) cand[nca++] = list[m];
                }
        qsort(cand, nca, sizeof(int), cmp_int);
        double xc[3]; float xcf[3];
        cell_centre(d, N, c, xc, xcf);
        double den = 0.0, num[4] = {0, 0, 0, 0};
        for (int m = 0; m < nca; ++m) {
            int i = cand[m];
            double q;
            if (!in_support(D, &rec[i], xc, xcf, &q)) continue;
            double w = rec[i].pref * exp(-0.5 * q);
            den += w;
            for (int a = 0; a < 1 + d; ++a) num[a] += w * rec[i].a[a];
        }
        double scale = D->per_cell ? V : 1.0;
        S_mass[o] = den > 0.0 ? -num[0] / den * scale : 0.0;
        for (int a = 0; a < d; ++a) S_mom[o * d + a] = den > 0.0 ? -num[1 + a] / den * scale : 0.0;
        Dsum[o] = den;
    }
    free(cand);
    }
    free(keys); free(start); free(list); free(fill); free(rec);
    return 0;
}

/* Host threads used by the loops above (1 when built without OpenMP). */
void ora_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int ora_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Audit of the single-precision truncation decision (test support): for each
 * listed cell, every candidate pair of the cell list is decided twice -- q <= 9
 * in double, and on the single-precision operands (D->fp32_decision must be 1)
 * -- and the pairs where the two disagree are recorded (list position of the
 * cell, droplet, q in double), up to max_out of them.  *n_pairs receives the
 * number of candidate pairs inside the double-precision support.  Returns the
 * number of disagreeing pairs. */
long ora_decision_audit(const ora_dep* D, int n, const double* x, const double* J, const double* acc,
                        const int* status, const int* batch, const double* n0, const double* h0,
                        long n_out, const long* cells, long max_out, long* out_cell, int* out_drop,
                        double* out_q, long* n_pairs)
{
    int d = D->dim, N = D->N;
    long nc = (d == 2) ? (long)N * N : (long)N * N * N;
    uint32_t* keys = (uint32_t*)malloc(sizeof(uint32_t) * (n > 0 ? n : 1));
    ora_cell_keys(d, N, n, x, status, 0, keys);
    long* start = (long*)calloc(nc + 1, sizeof(long));
    int* list = (int*)malloc(sizeof(int) * (n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) if (keys[i] != 0xFFFFFFFFu) start[keys[i] + 1]++;
    for (long c = 0; c < nc; ++c) start[c + 1] += start[c];
    long* fill = (long*)malloc(sizeof(long) * nc);
    memcpy(fill, start, sizeof(long) * nc);
    for (int i = 0; i < n; ++i) if (keys[i] != 0xFFFFFFFFu) list[fill[keys[i]]++] = i;
    ora_rec* rec = (ora_rec*)malloc(sizeof(ora_rec) * (n > 0 ? n : 1));
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i)
        if (keys[i] != 0xFFFFFFFFu)
            ora_record(D, x + (long)i * d, J + (long)i * d * d, acc + (long)i * (1 + d),
                       n0[batch[i]], h0[batch[i]], D->fold ? D->fold[i] : 0, &rec[i]);
    int R = (int)floor(3.0 * D->h_max * N + 0.5) + 1;
    long found = 0, inside = 0;
    for (long o = 0; o < n_out; ++o) {
        long c = cells[o];
        int ci[3] = {0, 0, 0};
        long r = c;
        for (int a = 0; a < d; ++a) { ci[a] = (int)(r % N); r /= N; }
        int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
        for (int a = 0; a < d; ++a) {
            lo[a] = ci[a] - R < 0 ? 0 : ci[a] - R;
            hi[a] = ci[a] + R > N - 1 ? N - 1 : ci[a] + R;
        }
        double xc[3]; float xcf[3];
        cell_centre(d, N, c, xc, xcf);
        for (int kz = lo[2]; kz <= hi[2]; ++kz)
            for (int ky = lo[1]; ky <= hi[1]; ++ky)
                for (int kx = lo[0]; kx <= hi[0]; ++kx) {
                    long b = kx + (long)N * ky + (long)N * N * kz;
                    for (long m = start[b]; m < start[b + 1]; ++m) {
                        int i = list[m];
                        double q;
                        int dec32 = in_support(D, &rec[i], xc, xcf, &q);
                        int dec64 = q <= 9.0;
                        inside += dec64;
                        if (dec32 != dec64) {
                            if (found < max_out) { out_cell[found] = o; out_drop[found] = i; out_q[found] = q; }
                            ++found;
                        }
                    }
                }
    }
    *n_pairs = inside;
    free(keys); free(start); free(list); free(fill); free(rec);
    return found;
}

/* Kernel of one droplet evaluated at every cell centre: the paper's weight
 * (normalised = 0) or the unit-mass Gaussian (normalised = 1, i.e. divided by
 * (2 pi)^{d/2} h^d, resp. (2 pi)^{d/2} det(Sigma)^{1/2}), truncated at q <= 9.
 * Used by the kernel-normalisation checks. */
void ora_kernel_on_cells(const ora_dep* D, const double* x, const double* J, double n0, double h0,
                         int normalised, double* w_out)
{
    int d = D->dim, N = D->N;
    long nc = (d == 2) ? (long)N * N : (long)N * N * N;
    double acc0[4] = {0, 0, 0, 0};
    ora_rec r;
    ora_record(D, x, J, acc0, n0, h0, 0, &r);
    double norm = 1.0;
    if (normalised) {
        double c2pi = pow(2.0 * ORA_PI, 0.5 * d);
        norm = (D->kernel == 0) ? 1.0 / (c2pi * pow(r.h, d) * r.pref) : 1.0 / c2pi;
    }
    for (long c = 0; c < nc; ++c) {
        double xc[3]; float xcf[3];
        cell_centre(d, N, c, xc, xcf);
        double q;
        w_out[c] = in_support(D, &r, xc, xcf, &q) ? r.pref * exp(-0.5 * q) * norm : 0.0;
    }
}

/* Per-droplet record values for tests: n, det J, h (or sqrt of the capped trace), pref. */
void ora_records(const ora_dep* D, int n, const double* x, const double* J, const double* acc,
                 const int* batch, const double* n0, const double* h0, double* out /* n x 4 */)
{
    int d = D->dim;
    for (int i = 0; i < n; ++i) {
        ora_rec r;
        ora_record(D, x + (long)i * d, J + (long)i * d * d, acc + (long)i * (1 + d),
                   n0[batch[i]], h0[batch[i]], D->fold ? D->fold[i] : 0, &r);
        out[i * 4 + 0] = r.n;
        out[i * 4 + 1] = r.detJ;
        out[i * 4 + 2] = r.h;
        out[i * 4 + 3] = r.pref;
    }
}

/* ------------------------------------------------------------------------ */
/* PSI-CELL box count (Eqs. 10-11)                                           */
/* ------------------------------------------------------------------------ */

/* counts_c = number of active parcels in cell c;
 * S_mass = -(1/V) sum w a_m,  S_mom = -(1/V) sum w a_mom over the parcels of the
 * cell in ascending index, a = acc / T_window, w = real droplets per parcel of
 * the parcel's release.  per_cell drops the 1/V. */
int ora_psicell(const ora_dep* D, int n, const double* x, const double* acc, const int* status,
                const int* batch, const double* w, int fp32_keys,
                uint32_t* counts, double* S_mass, double* S_mom)
{
    int d = D->dim, N = D->N;
    long nc = (d == 2) ? (long)N * N : (long)N * N * N;
    uint32_t* keys = (uint32_t*)malloc(sizeof(uint32_t) * (n > 0 ? n : 1));
    ora_cell_keys(d, N, n, x, status, fp32_keys, keys);
    for (long c = 0; c < nc; ++c) {
        counts[c] = 0; S_mass[c] = 0.0;
        for (int a = 0; a < d; ++a) S_mom[c * d + a] = 0.0;
    }
    double V = cell_volume(D);
    double scale = D->per_cell ? 1.0 : 1.0 / V;
    for (int i = 0; i < n; ++i) {
        if (keys[i] == 0xFFFFFFFFu) continue;
        long c = keys[i];
        double wi = w[batch[i]];
        counts[c] += 1;
        S_mass[c] += -scale * wi * acc[(long)i * (1 + d)] / D->window_dt;
        for (int a = 0; a < d; ++a)
            S_mom[c * d + a] += -scale * wi * acc[(long)i * (1 + d) + 1 + a] / D->window_dt;
    }
    free(keys);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Cloud-In-Cell deposit (the C^1 alternative to PSI-CELL named in Sec. 1)    */
/* ------------------------------------------------------------------------ */

/* Tent weight of a parcel at x for the cell centred at xc: the overlap of a
 * cell-sized cloud around the parcel with the cell, prod_a max(0, 1 - |x_a -
 * xc_a| N) (reading: the paper's CIC interpolates to the corners of the cell
 * that holds the parcel; with cell-centred sources those corners are the cell
 * centres around the parcel, the corners of its dual cell). */
static double cic_weight(int d, int N, const double* x, const double* xc)
{
    double w = 1.0;
    for (int a = 0; a < d; ++a) {
        double t = 1.0 - fabs(x[a] - xc[a]) * N;
        if (t <= 0.0) return 0.0;
        w *= t;
    }
    return w;
}

/* Box counts of a parcel cloud: counts_c = parcels whose cell key is c, the
 * key formed in double or, with fp32_keys, in single precision (R18). */
static void box_counts(int d, int N, int n, const double* x, const int* status, int fp32_keys, uint32_t* counts)
{
    long nc = (d == 2) ? (long)N * N : (long)N * N * N;
    uint32_t* keys = (uint32_t*)malloc(sizeof(uint32_t) * (n > 0 ? n : 1));
    ora_cell_keys(d, N, n, x, status, fp32_keys, keys);
    for (long c = 0; c < nc; ++c) counts[c] = 0;
    for (int i = 0; i < n; ++i) if (keys[i] != 0xFFFFFFFFu) counts[keys[i]] += 1;
    free(keys);
}

/* S_c = -(1/V) sum_i W(x_i, x_c) w_i acc_i / T over active parcels inside
 * [0,1]^d, in ascending parcel index (brute force over every parcel), and
 * counts_c = parcels whose cell key is c (the box count, as PSI-CELL).
 * Weight of centres outside the mesh is dropped (no redistribution). */
int ora_cic(const ora_dep* D, int n, const double* x, const double* acc, const int* status, const int* batch,
            const double* w, int fp32_keys, uint32_t* counts, double* S_mass, double* S_mom)
{
    int d = D->dim, N = D->N;
    long nc = (d == 2) ? (long)N * N : (long)N * N * N;
    uint32_t* keys = (uint32_t*)malloc(sizeof(uint32_t) * (n > 0 ? n : 1));
    ora_cell_keys(d, N, n, x, status, 0, keys);
    double scale = D->per_cell ? 1.0 : 1.0 / cell_volume(D);
    box_counts(d, N, n, x, status, fp32_keys, counts);
#pragma omp parallel for schedule(dynamic, 64)
    for (long c = 0; c < nc; ++c) {
        double xc[3]; float xcf[3];
        cell_centre(d, N, c, xc, xcf);
        double s[4] = {0, 0, 0, 0};
        for (int i = 0; i < n; ++i) {
            if (keys[i] == 0xFFFFFFFFu) continue;
            double W = cic_weight(d, N, x + (long)i * d, xc);
            if (W == 0.0) continue;
            for (int a = 0; a <= d; ++a) s[a] += W * w[batch[i]] * acc[(long)i * (1 + d) + a] / D->window_dt;
        }
        S_mass[c] = -scale * s[0];
        for (int a = 0; a < d; ++a) S_mom[c * d + a] = -scale * s[1 + a];
    }
    free(keys);
    return 0;
}

/* The same deposit through the cell list: a cell's contributors are the parcels
 * binned in the 3^d cells around it (W vanishes beyond one cell), taken in
 * ascending index; bit-identical to ora_cic. */
int ora_cic_celllist(const ora_dep* D, int n, const double* x, const double* acc, const int* status,
                     const int* batch, const double* w, int fp32_keys, uint32_t* counts, double* S_mass,
                     double* S_mom)
{
    int d = D->dim, N = D->N;
    long nc = (d == 2) ? (long)N * N : (long)N * N * N;
    uint32_t* keys = (uint32_t*)malloc(sizeof(uint32_t) * (n > 0 ? n : 1));
    ora_cell_keys(d, N, n, x, status, 0, keys);
    long* start = (long*)calloc(nc + 1, sizeof(long));
    int* list = (int*)malloc(sizeof(int) * (n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) if (keys[i] != 0xFFFFFFFFu) start[keys[i] + 1]++;
    for (long c = 0; c < nc; ++c) start[c + 1] += start[c];
    box_counts(d, N, n, x, status, fp32_keys, counts);
    long* fill = (long*)malloc(sizeof(long) * nc);
    memcpy(fill, start, sizeof(long) * nc);
    for (int i = 0; i < n; ++i) if (keys[i] != 0xFFFFFFFFu) list[fill[keys[i]]++] = i;
    double scale = D->per_cell ? 1.0 : 1.0 / cell_volume(D);
#pragma omp parallel
    {
    int* cand = (int*)malloc(sizeof(int) * (n > 0 ? n : 1));
#pragma omp for schedule(dynamic, 64)
    for (long c = 0; c < nc; ++c) {
        int ci[3] = {0, 0, 0};
        long r = c;
        for (int a = 0; a < d; ++a) { ci[a] = (int)(r % N); r /= N; }
        int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
        for (int a = 0; a < d; ++a) {
            lo[a] = ci[a] > 0 ? ci[a] - 1 : 0;
            hi[a] = ci[a] < N - 1 ? ci[a] + 1 : N - 1;
        }
        int nca = 0;
        for (int kz = lo[2]; kz <= hi[2]; ++kz)
            for (int ky = lo[1]; ky <= hi[1]; ++ky)
                for (int kx = lo[0]; kx <= hi[0]; ++kx) {
                    long b = kx + (long)N * ky + (long)N * N * kz;
                    for (long m = start[b]; m < start[b + 1]; ++m) cand[nca++] = list[m];
                }
        qsort(cand, nca, sizeof(int), cmp_int);
        double xc[3]; float xcf[3];
        cell_centre(d, N, c, xc, xcf);
        double s[4] = {0, 0, 0, 0};
        for (int m = 0; m < nca; ++m) {
            int i = cand[m];
            double W = cic_weight(d, N, x + (long)i * d, xc);
            if (W == 0.0) continue;
            for (int a = 0; a <= d; ++a) s[a] += W * w[batch[i]] * acc[(long)i * (1 + d) + a] / D->window_dt;
        }
        S_mass[c] = -scale * s[0];
        for (int a = 0; a < d; ++a) S_mom[c * d + a] = -scale * s[1 + a];
    }
    free(cand);
    }
    free(keys); free(start); free(list); free(fill);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Learned bandwidth correction (no counterpart in the paper)                */
/* ------------------------------------------------------------------------ */
/*
 * A small MLP g maps per-droplet features to a correction of the smoothing
 * length of Eq. 15: h = clamp(h0 |det J|^p * exp(clip(g(f), -2, 2)), h_min, h_max).
 * g is 6 -> 64 -> 64 -> 64 -> 1 with SiLU after the three hidden layers.
 * Parameters are single-precision masters; the forward uses them rounded to
 * bfloat16 (round to nearest even), the biases unrounded, and rounds the
 * inputs of the first three layers to bfloat16 as a tensor-core forward does.
 * Arithmetic here is double precision.
 *
 * Features (readings of "local J invariants, n and neighbour spacing"):
 *   f0 = ln ||J||_F^2 / 8                  first invariant of J^T J
 *   f1 = ln ||cof J||_F^2 / 8 (3D), ln det(J)^2 / 8 (2D)   second invariant
 *   f2 = ln |det J| / 8
 *   f3 = ln n / 8,  n = n0 / max(|det J|, 1e-12)           (Eq. 6)
 *   f4 = ln(h0 |det J|^(1/d) / dx) / 4      Lagrangian seed spacing over the cell size
 *   f5 = min(|det J|, 4) / 4
 * with ln taken of max(x, 1e-30).
 *
 * Parameter layout (ORA_MLP_NPARAM floats): W1[64][6], b1[64], W2[64][64],
 * b2[64], W3[64][64], b3[64], W4[64], b4 (rows are output units).
 */
#define ORA_MLP_IN 6
#define ORA_MLP_H 64
#define ORA_MLP_NPARAM (ORA_MLP_H * ORA_MLP_IN + ORA_MLP_H + 2 * (ORA_MLP_H * ORA_MLP_H + ORA_MLP_H) + ORA_MLP_H + 1)

static const int ORA_OFF_W1 = 0;
static const int ORA_OFF_B1 = ORA_MLP_H * ORA_MLP_IN;
static const int ORA_OFF_W2 = ORA_MLP_H * ORA_MLP_IN + ORA_MLP_H;
static const int ORA_OFF_B2 = ORA_MLP_H * ORA_MLP_IN + ORA_MLP_H + ORA_MLP_H * ORA_MLP_H;
static const int ORA_OFF_W3 = ORA_MLP_H * ORA_MLP_IN + 2 * ORA_MLP_H + ORA_MLP_H * ORA_MLP_H;
static const int ORA_OFF_B3 = ORA_MLP_H * ORA_MLP_IN + 2 * ORA_MLP_H + 2 * ORA_MLP_H * ORA_MLP_H;
static const int ORA_OFF_W4 = ORA_MLP_H * ORA_MLP_IN + 3 * ORA_MLP_H + 2 * ORA_MLP_H * ORA_MLP_H;
static const int ORA_OFF_B4 = ORA_MLP_H * ORA_MLP_IN + 4 * ORA_MLP_H + 2 * ORA_MLP_H * ORA_MLP_H;

int ora_mlp_nparam(void) { return ORA_MLP_NPARAM; }

/* bfloat16 value of a float: keep the top 16 bits, rounding to nearest even */
static int g_mlp_exact;
static double bf16_of_float(float x)
{
    if (g_mlp_exact) return (double)x;
    uint32_t u;
    memcpy(&u, &x, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);
    u &= 0xFFFF0000u;
    float r;
    memcpy(&r, &u, 4);
    return (double)r;
}

/* bfloat16 value nearest to a double (ties to even), and the spacing of the
 * bfloat16 numbers around it; finite normal range only */
static double bf16_of_double(double x, double* spacing)
{
    if (g_mlp_exact) { if (spacing) *spacing = 0.0; return x; }
    if (x == 0.0) { if (spacing) *spacing = ldexp(1.0, -133); return 0.0; }
    int e;
    frexp(x, &e);                          /* |x| in [2^(e-1), 2^e) */
    double ulp = ldexp(1.0, e - 8);        /* 8 significant bits */
    double q = x / ulp;
    double r = nearbyint(q);               /* default rounding mode: to nearest even */
    if (spacing) *spacing = ulp;
    return r * ulp;
}

/* distance from x to the nearest rounding boundary (midpoint between two
 * consecutive bfloat16 numbers) */
static double bf16_boundary_distance(double x)
{
    double sp;
    double r = bf16_of_double(x, &sp);
    double d = fabs(fabs(x - r) - 0.5 * sp);
    return d;
}

static double silu(double z) { return z / (1.0 + exp(-z)); }
static double silu_d(double z) { double s = 1.0 / (1.0 + exp(-z)); return s * (1.0 + z * (1.0 - s)); }

void ora_mlp_features(int d, const double* J, double n0, double h0, double dx, double* f)
{
    double I1 = 0.0;
    for (int q = 0; q < d * d; ++q) I1 += J[q] * J[q];
    double det = det_d(d, J);
    double ad = fabs(det);
    double I2;
    if (d == 2) {
        I2 = det * det;
    } else {
        I2 = 0.0;   /* squared 2x2 minors: the Frobenius norm of the cofactor matrix */
        for (int r0 = 0; r0 < 3; ++r0)
            for (int r1 = r0 + 1; r1 < 3; ++r1)
                for (int c0 = 0; c0 < 3; ++c0)
                    for (int c1 = c0 + 1; c1 < 3; ++c1) {
                        double m = J[r0 * 3 + c0] * J[r1 * 3 + c1] - J[r0 * 3 + c1] * J[r1 * 3 + c0];
                        I2 += m * m;
                    }
    }
    double n = n0 / (ad > 1e-12 ? ad : 1e-12);
    f[0] = log(I1 > 1e-30 ? I1 : 1e-30) / 8.0;
    f[1] = log(I2 > 1e-30 ? I2 : 1e-30) / 8.0;
    f[2] = log(ad > 1e-30 ? ad : 1e-30) / 8.0;
    f[3] = log(n > 1e-30 ? n : 1e-30) / 8.0;
    double sp = h0 * pow(ad, 1.0 / d) / dx;
    f[4] = log(sp > 1e-30 ? sp : 1e-30) / 4.0;
    f[5] = (ad < 4.0 ? ad : 4.0) / 4.0;
}

/* Rounds v to bfloat16 and returns, in *dev, a bound on how far a forward
 * that computed v with error at most e and rounded it could be from the
 * rounded value: 0 when no rounding boundary lies within e of v. */
/* 1: no bfloat16 rounding anywhere (the network in plain double precision,
 * for finite-difference checks of the gradient) */
void ora_mlp_set_exact(int exact) { g_mlp_exact = exact; }

static double round_with_bound(double v, double e, double* dev)
{
    if (g_mlp_exact) { *dev = e; return v; }
    double sp;
    double r = bf16_of_double(v, &sp);
    *dev = (bf16_boundary_distance(v) > e) ? 0.0 : e + sp;
    return r;
}

/*
 * Forward pass.  Returns c = g(f).  If bound != NULL it receives a bound on
 * |c_single - c| for a forward that evaluates the same network with
 * single-precision accumulation (relative error of each dot product of K terms
 * at most 2 K 2^-24 of the sum of |terms|), a single-precision SiLU (error at
 * most 2^-20 (|z| + |silu(z)|)) and features with absolute errors fe[k]
 * (NULL: 1e-6 (1 + |f|)): the bound propagates these through the layers and
 * adds one bfloat16 spacing wherever a rounding boundary lies within the
 * propagated error.  act (optional, 3 x 64) receives the post-SiLU values
 * before rounding and zs (optional, 3 x 64) the pre-activations.
 */
double ora_mlp_forward(const float* P, const double* f, const double* fe, double* bound, double* act, double* zs)
{
    const int H = ORA_MLP_H;
    double a0[ORA_MLP_IN], e0[ORA_MLP_IN];
    for (int k = 0; k < ORA_MLP_IN; ++k) {
        double ef = fe ? fe[k] : 1e-6 * (1.0 + fabs(f[k]));
        a0[k] = round_with_bound(f[k], ef, &e0[k]);
    }
    double a[ORA_MLP_H], ea[ORA_MLP_H], nxt[ORA_MLP_H], en[ORA_MLP_H];
    const int K1 = ORA_MLP_IN;
    for (int j = 0; j < H; ++j) {
        double z = 0.0, s_abs = 0.0, prop = 0.0;
        for (int k = 0; k < K1; ++k) {
            double w = bf16_of_float(P[ORA_OFF_W1 + j * K1 + k]);
            z += w * a0[k];
            s_abs += fabs(w * a0[k]);
            prop += fabs(w) * e0[k];
        }
        z += (double)P[ORA_OFF_B1 + j];
        double ez = prop + 2.0 * (K1 + 1) * ldexp(s_abs + fabs(z), -24);
        double p = silu(z);
        double ep = 1.1 * ez + ldexp(fabs(z) + fabs(p), -20);
        if (zs) zs[j] = z;
        if (act) act[j] = p;
        a[j] = round_with_bound(p, ep, &ea[j]);
    }
    for (int layer = 0; layer < 2; ++layer) {
        const int ow = layer == 0 ? ORA_OFF_W2 : ORA_OFF_W3;
        const int ob = layer == 0 ? ORA_OFF_B2 : ORA_OFF_B3;
        for (int j = 0; j < H; ++j) {
            double z = 0.0, s_abs = 0.0, prop = 0.0;
            for (int k = 0; k < H; ++k) {
                double w = bf16_of_float(P[ow + j * H + k]);
                z += w * a[k];
                s_abs += fabs(w * a[k]);
                prop += fabs(w) * ea[k];
            }
            z += (double)P[ob + j];
            double ez = prop + 2.0 * (H + 1) * ldexp(s_abs + fabs(z), -24);
            double p = silu(z);
            double ep = 1.1 * ez + ldexp(fabs(z) + fabs(p), -20);
            if (zs) zs[(layer + 1) * H + j] = z;
            if (act) act[(layer + 1) * H + j] = p;
            if (layer == 0) {
                nxt[j] = round_with_bound(p, ep, &en[j]);
            } else {
                nxt[j] = p;            /* the last hidden layer feeds a single-precision dot product */
                en[j] = ep;
            }
        }
        memcpy(a, nxt, sizeof(a));
        memcpy(ea, en, sizeof(ea));
    }
    double c = 0.0, s_abs = 0.0, prop = 0.0;
    for (int k = 0; k < H; ++k) {
        double w = bf16_of_float(P[ORA_OFF_W4 + k]);
        c += w * a[k];
        s_abs += fabs(w * a[k]);
        prop += fabs(w) * ea[k];
    }
    c += (double)P[ORA_OFF_B4];
    if (bound) *bound = prop + 2.0 * (H + 1) * ldexp(s_abs + fabs(c), -24);
    return c;
}

/*
 * Gradient of c = g(f) with respect to the master parameters, times dLdc,
 * added to grad (ORA_MLP_NPARAM doubles).  The bfloat16 roundings are treated
 * as the identity (straight-through), so the gradient is that of the network
 * evaluated with the rounded weights and activations.
 */
void ora_mlp_backward(const float* P, const double* f, double dLdc, double* grad)
{
    const int H = ORA_MLP_H;
    double z[3 * ORA_MLP_H], p[3 * ORA_MLP_H];
    ora_mlp_forward(P, f, NULL, NULL, p, z);
    double a0[ORA_MLP_IN];
    for (int k = 0; k < ORA_MLP_IN; ++k) a0[k] = bf16_of_double(f[k], NULL);
    double a1[ORA_MLP_H], a2[ORA_MLP_H], a3[ORA_MLP_H];
    for (int j = 0; j < H; ++j) {
        a1[j] = bf16_of_double(p[j], NULL);
        a2[j] = bf16_of_double(p[H + j], NULL);
        a3[j] = p[2 * H + j];
    }
    /* layer 4 */
    double d3[ORA_MLP_H];
    for (int k = 0; k < H; ++k) {
        grad[ORA_OFF_W4 + k] += dLdc * a3[k];
        d3[k] = dLdc * bf16_of_float(P[ORA_OFF_W4 + k]) * silu_d(z[2 * H + k]);
    }
    grad[ORA_OFF_B4] += dLdc;
    /* layer 3: z3 = W3 a2 + b3 */
    double d2[ORA_MLP_H];
    for (int k = 0; k < H; ++k) d2[k] = 0.0;
    for (int j = 0; j < H; ++j) {
        grad[ORA_OFF_B3 + j] += d3[j];
        for (int k = 0; k < H; ++k) {
            grad[ORA_OFF_W3 + j * H + k] += d3[j] * a2[k];
            d2[k] += d3[j] * bf16_of_float(P[ORA_OFF_W3 + j * H + k]);
        }
    }
    for (int k = 0; k < H; ++k) d2[k] *= silu_d(z[H + k]);
    /* layer 2: z2 = W2 a1 + b2 */
    double d1[ORA_MLP_H];
    for (int k = 0; k < H; ++k) d1[k] = 0.0;
    for (int j = 0; j < H; ++j) {
        grad[ORA_OFF_B2 + j] += d2[j];
        for (int k = 0; k < H; ++k) {
            grad[ORA_OFF_W2 + j * H + k] += d2[j] * a1[k];
            d1[k] += d2[j] * bf16_of_float(P[ORA_OFF_W2 + j * H + k]);
        }
    }
    for (int k = 0; k < H; ++k) d1[k] *= silu_d(z[k]);
    /* layer 1: z1 = W1 a0 + b1 */
    for (int j = 0; j < H; ++j) {
        grad[ORA_OFF_B1 + j] += d1[j];
        for (int k = 0; k < ORA_MLP_IN; ++k) grad[ORA_OFF_W1 + j * ORA_MLP_IN + k] += d1[j] * a0[k];
    }
}

/* Batch helpers for tests: c (and its bound) for n feature rows. */
void ora_mlp_forward_batch(const float* P, int n, const double* F, const double* FE, double* c, double* bound)
{
    for (int i = 0; i < n; ++i)
        c[i] = ora_mlp_forward(P, F + (long)i * ORA_MLP_IN, FE ? FE + (long)i * ORA_MLP_IN : NULL,
                               bound ? &bound[i] : NULL, NULL, NULL);
}

/*
 * Training loss of the learned correction and its gradient.
 * At the listed training cells c and for each source component k (mass, then
 * momentum):
 *   L = 1/(1+d) sum_k sum_c (S_kc - T_kc)^2 / sum_c T_kc^2,
 * S the Nadaraya-Watson sources of the cloud with the corrected bandwidth, T
 * the targets (n_train x (1+d)).  dS_kc/dw_ic = -(a_ki + S_kc)/D_c, and
 *  - spherical kernel, w_ic = exp(-q/2)/h_i, q = r^2/h_i^2, dh_i/dc_i = h_i:
 *      dw_ic/dc_i = w_ic (q - 1);
 *  - J-scaled kernel, w_ic = det(Sigma_i)^(-1/2) exp(-q/2), q = r' P_i r,
 *    P_i = Sigma_i^-1, Sigma_i = e^(2c_i) A_i + h_min^2 I (trace cap inactive),
 *    so dSigma/dc = 2 (Sigma - h_min^2 I):
 *      dq/dc = -r' P dSigma/dc P r = -2 (q - h_min^2 |P r|^2),
 *      d log det(Sigma)^(-1/2)/dc = -tr(P (Sigma - h_min^2 I)) = -(d - h_min^2 tr P),
 *      dw_ic/dc_i = w_ic ((q - h_min^2 |P r|^2) - (d - h_min^2 tr P));
 * so dL/dc_i = -sum_c (dw_ic/dc_i) sum_k g_kc (a_ki + S_kc)/D_c with
 * g_kc = dL/dS_kc; the truncation edge is held fixed.  The gradient with
 * respect to the parameters follows by ora_mlp_backward.  grad may be NULL.
 */
static double dw_dc(const ora_dep* D, const ora_rec* r, const double* xc, double q, double w)
{
    int d = D->dim;
    if (D->kernel == 0) return w * (q - 1.0);
    double rv[3], pr[3], pr2 = 0.0, trP = 0.0;
    for (int a = 0; a < d; ++a) rv[a] = xc[a] - r->x[a];
    for (int i = 0; i < d; ++i) {
        pr[i] = 0.0;
        for (int k = 0; k < d; ++k) pr[i] += r->P[i * d + k] * rv[k];
        pr2 += pr[i] * pr[i];
        trP += r->P[i * d + i];
    }
    double h2 = D->h_min * D->h_min;
    return w * ((q - h2 * pr2) - (d - h2 * trP));
}

int ora_learn_loss_grad(const ora_dep* D, int n, const double* x, const double* J, const double* acc,
                        const int* status, const int* batch, const double* n0, const double* h0,
                        long n_train, const long* cells, const double* target, double* loss, double* grad)
{
    int d = D->dim;
    if (!D->mlp) return -1;
    ora_rec* rec = (ora_rec*)malloc(sizeof(ora_rec) * (n > 0 ? n : 1));
    int* use = (int*)malloc(sizeof(int) * (n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) {
        use[i] = contributes(d, x + (long)i * d, status[i]);
        if (use[i])
            ora_record(D, x + (long)i * d, J + (long)i * d * d, acc + (long)i * (1 + d),
                       n0[batch[i]], h0[batch[i]], D->fold ? D->fold[i] : 0, &rec[i]);
    }
    double* S = (double*)calloc((size_t)n_train * (1 + d), sizeof(double));
    double* Dc = (double*)calloc((size_t)n_train, sizeof(double));
    for (long o = 0; o < n_train; ++o) {
        double xc[3]; float xcf[3];
        cell_centre(d, D->N, cells[o], xc, xcf);
        double den = 0.0, num[4] = {0, 0, 0, 0};
        for (int i = 0; i < n; ++i) {
            if (!use[i]) continue;
            double q;
            if (!in_support(D, &rec[i], xc, xcf, &q)) continue;
            double w = rec[i].pref * exp(-0.5 * q);
            den += w;
            for (int a = 0; a < 1 + d; ++a) num[a] += w * rec[i].a[a];
        }
        Dc[o] = den;
        for (int a = 0; a < 1 + d; ++a) S[o * (1 + d) + a] = den > 0.0 ? -num[a] / den : 0.0;
    }
    double L = 0.0, norm[4] = {0, 0, 0, 0};
    for (long o = 0; o < n_train; ++o)
        for (int a = 0; a < 1 + d; ++a) norm[a] += target[o * (1 + d) + a] * target[o * (1 + d) + a];
    for (int a = 0; a < 1 + d; ++a) {
        double e = 0.0;
        for (long o = 0; o < n_train; ++o) {
            double r = S[o * (1 + d) + a] - target[o * (1 + d) + a];
            e += r * r;
        }
        L += norm[a] > 0.0 ? e / norm[a] : 0.0;
    }
    L /= (1 + d);
    *loss = L;
    if (grad) {
        for (int i = 0; i < n; ++i) {
            if (!use[i] || !rec[i].dh_dc) continue;
            double dLdc = 0.0;
            for (long o = 0; o < n_train; ++o) {
                if (!(Dc[o] > 0.0)) continue;
                double xc[3]; float xcf[3];
                cell_centre(d, D->N, cells[o], xc, xcf);
                double q;
                if (!in_support(D, &rec[i], xc, xcf, &q)) continue;
                double w = rec[i].pref * exp(-0.5 * q);
                double acc_k = 0.0;
                for (int a = 0; a < 1 + d; ++a) {
                    if (!(norm[a] > 0.0)) continue;
                    double g = 2.0 * (S[o * (1 + d) + a] - target[o * (1 + d) + a]) / (norm[a] * (1 + d));
                    acc_k += g * (rec[i].a[a] + S[o * (1 + d) + a]);
                }
                dLdc += -dw_dc(D, &rec[i], xc, q, w) * acc_k / Dc[o];
            }
            if (dLdc != 0.0) ora_mlp_backward(D->mlp, rec[i].f, dLdc, grad);
        }
    }
    free(rec); free(use); free(S); free(Dc);
    return 0;
}

/* Per-droplet learned correction of the records (tests): c and the flag dh/dc != 0. */
void ora_learn_records(const ora_dep* D, int n, const double* x, const double* J, const double* acc,
                       const int* batch, const double* n0, const double* h0, double* c, int* active, double* h)
{
    int d = D->dim;
    for (int i = 0; i < n; ++i) {
        ora_rec r;
        ora_record(D, x + (long)i * d, J + (long)i * d * d, acc + (long)i * (1 + d), n0[batch[i]], h0[batch[i]],
                   D->fold ? D->fold[i] : 0, &r);
        c[i] = r.c;
        active[i] = r.dh_dc;
        h[i] = r.h;
    }
}
