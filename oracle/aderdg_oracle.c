/*
 * Plain FP64 CPU oracle of the unlimited ADER-DG scheme of Dumbser, Fambri,
 * Tavelli, Bader and Weinzierl (2018), "Efficient implementation of ADER
 * discontinuous Galerkin schemes for a scalable hyperbolic PDE engine".
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file.  It shares no code, header, table or constant generator
 * with the CUDA library; it is meant to be slow and obviously correct.
 *
 * What it computes (section / equation of the paper):
 *   - nodal tensor-product basis on N+1 Gauss-Legendre nodes of [0,1]
 *     (Sec. 2.1, ansatz for u_h)
 *   - space-time predictor: weak form integrated by parts in time
 *     (Sec. 2.2, eq. pde.st2), solved by a discrete Picard iteration started
 *     from the trivial guess q = u(t^n); discrete derivatives are the nodal
 *     derivative matrix D (eq. D_kl) applied dimension by dimension
 *   - corrector (Sec. 2.1, eq. pde.nc.gw2): diagonal mass, volume integrals
 *     of grad(Phi).F(q_h), Phi B(q_h).grad(q_h) and Phi S(q_h), face
 *     integral of the path-conservative Rusanov fluctuations (eq. pc.scheme
 *     with the straight-segment path and a three-point Gauss-Legendre rule
 *     for the path integral, eq. rusanov) on time-averaged traces
 *   - CFL time step dt = alpha / sum_d lambda_d^max / dx_d (Sec. 3, CFL eq.)
 *   - the a posteriori subcell finite-volume limiter (Sec. 2.3): detection
 *     on the candidate (non-finite values, Euler positivity, a relaxed
 *     discrete maximum principle on subcell averages), a second-order
 *     finite-volume step of the troubled elements on (2N+1)^d subcells,
 *     least-squares reconstruction of the DG polynomial, and the matching
 *     face fluxes in the unlimited neighbours (readings R25-R29; with
 *     non-conservative products and sources, eq. pde.nc.fv), optionally
 *     with the limited elements' subcell averages kept between steps (R35)
 *   - PDEs: linear advection with an optional linear reaction source
 *     S = -kappa q, Euler (Sec. 3.1, eq. euler, ideal gas), the
 *     velocity-stress linear elasticity system obtained from Sec. 3.2 with
 *     alpha = 1 and constant rho, lambda, mu (conservative form), and the
 *     diffuse-interface elasticity system of Sec. 3.2 itself (purely
 *     non-conservative, material parameters and alpha in the state)
 *
 * Readings of points where the paper is silent or ambiguous (listed in the
 * design notes as well):
 *   R1 the predictor's right-hand side is -div F (moving div F from the
 *      left-hand side of eq. pde to the right; cf. the L operator of Sec. 2.2)
 *   R2 the flux divergence in the predictor is the nodal derivative of the
 *      nodal flux interpolant (eq. D_kl applied to flux DOFs)
 *   R3 a fixed number of Picard iterations P (default N+1); picard < 0
 *      iterates to convergence instead (used by checks only)
 *   R5 the Riemann solver acts on time averages: qbar and Fbar_d are
 *      extrapolated to the faces; Fbar at the face is the extrapolation of
 *      the volume Fbar_d, not F of the extrapolated qbar
 *   R6 s_max is taken per face node from the time-averaged traces
 *   R7 alpha defaults to 0.9 x the von Neumann limit of the scheme (the
 *      paper's alpha < 1/(2N+1) is necessary only; 0.9/(2N+1) is unstable
 *      for N >= 3); the last step is clipped to t_end
 *   R19 diffuse-interface elasticity: state (sigma, w = alpha v, alpha,
 *      lambda, mu, rho); the stress equation's (1/alpha) grad(alpha v) is
 *      the gradient of the state variable w, and v = w / alpha; alpha > 0
 *      everywhere (a vacuum is a small positive alpha); in 2D the
 *      plane-strain subsystem (sxx, syy, sxy, w1, w2) without szz
 *   R20 the dissipation matrix Theta = s_max I acts on the evolved
 *      variables only: the material parameters and alpha obey q_t = 0,
 *      which Rusanov dissipation of their jumps would violate
 *   R21 the path-conservative face term uses the time-averaged traces (as
 *      R5); the lower element of a face receives
 *      (fL + fR)/2 - Theta (qR - qL)/2 + J/2 and the upper one the same
 *      with -J/2, J = int_0^1 B_d(psi(s)) ds (qR - qL)
 *   R25 detection: a candidate element is troubled if a value is not
 *      finite, if (Euler) density or pressure is not positive at a node or
 *      in a subcell average, or if a subcell average leaves
 *      [lo - delta, hi + delta], lo / hi the extreme subcell averages of
 *      u^n over the element and its 2d face neighbours,
 *      delta = max(1e-4, 1e-3 (hi - lo))
 *   R26 the subcell scheme: MUSCL-Hancock with minmod slopes and the
 *      Rusanov flux, direction by direction (each face flux uses the two
 *      adjacent subcells' values and normal slopes, with the half-step
 *      evolution along that direction), ghost data two subcells deep from
 *      the face neighbours' u^n
 *   R27 an unlimited neighbour of a troubled element takes, on their common
 *      face, the subcell fluxes projected onto its face nodes
 *      (F(p) = sum_seg F_seg int_seg phi_p / w_p) instead of its DG flux
 *   R28 reconstruction: least squares from the (2N+1)^d subcell averages;
 *      with equal subcells it keeps the element's mass
 *   R29 the subcell scheme with B(Q) grad Q and S(Q) (eq. pde.nc.fv): the
 *      half-step of each face value adds -(dt/2h) B_d(w) s and (dt/2) S(w)
 *      (w the subcell average, s its minmod slope); a face gives the lower
 *      subcell the path-conservative fluctuation of the DG faces (R20) with
 *      +J/2 and the upper one that with -J/2; inside the subcell
 *      -(dt/h) B_d(w~) s is added, w~ the half-step centre along d; the
 *      source enters as dt S(w*), w* = w + the half-step changes of all
 *      directions + (dt/2) S(w); the material fields are kept as they were
 *   R30 coupling with B(Q) grad Q: an unlimited neighbour takes, per face
 *      node, the projected subcell fluctuation it receives plus the path
 *      integral J from its own DG trace to its own subcell state at that
 *      subcell face (with B the Jacobian of a flux this is R27: the flux
 *      difference between the two states of its own side)
 *   R35 kept subcell data (limiter mode 2): for an element the step that
 *      produced u^n limited, the subcell data at t^n (eq. subcellaverage)
 *      are the averages its subcell scheme produced, not those of their
 *      least-squares reconstruction; they enter the bounds, the subcell
 *      scheme and the coupling, and its CFL wave speeds come from them; a
 *      state may be given as the subcell averages of every element
 *
 * Layout: u[e][s][v] with v fastest, then x, y, z (s = sx + n*sy + n^2*sz);
 * space-time qhat[t][s][v] with time slowest (the AoS layout of Sec. 2.2).
 * Elements e = ex + Cx*(ey + Cy*ez).  All boundaries are periodic.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC (strict IEEE FP64,
 * no contraction into FMA).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAXN 10   /* n = N+1 <= 10 */
#define ORC_MAXM 13   /* variables */

typedef struct {
    int dim;          /* 1, 2 or 3 */
    int cells[3];     /* elements per dimension */
    double lo[3], hi[3];
    int N;            /* polynomial degree */
    int m;            /* number of variables */
    int pde;          /* 1 advection, 2 Euler, 3 elasticity, 4 diffuse-interface
                         elasticity */
    double prm[8];    /* advection: a_x a_y a_z kappa; Euler: gamma; elasticity:
                         rho lambda mu; diffuse interface: none (all in the state) */
    int picard;       /* > 0 fixed count, 0 -> default (see orc_picard_count),
                         < 0 -> to convergence */
    double alpha;     /* CFL coefficient; 0 -> default table (see orc_alpha) */
    int guess;        /* initial guess of the Picard iteration (Sec. 2.2):
                         0 trivial q = u(t^n); 1 second order u + tau L(u);
                         2 third order u + tau k1 + tau^2 (k2 - k1) / (2 dt);
                         3 extrapolation of the previous step's predictor
                           (orc_run; the first step, and single steps, use 2);
                         4 continuous Runge-Kutta (CERK) dense output, a
                           polynomial of degree min(5, max(3, N - 1)) in
                           time */
    int limiter;      /* 1: a posteriori subcell finite-volume limiter
                         (Sec. 2.3) after every step; 2: the same with the
                         limited elements' subcell averages kept (R35) */
} orc_cfg;

/* ------------------------------------------------------------------------ */
/* 1D basis (Sec. 2.1)                                                       */
/* ------------------------------------------------------------------------ */

/* Legendre polynomial P_n(y) and its derivative, by the three-term recurrence
 * (k+1) P_{k+1} = (2k+1) y P_k - k P_{k-1}. */
static void legendre(int n, double y, double *p, double *dp)
{
    double p0 = 1.0, p1 = y;
    if (n == 0) { *p = 1.0; *dp = 0.0; return; }
    for (int k = 1; k < n; ++k) {
        double p2 = ((2.0 * k + 1.0) * y * p1 - k * p0) / (k + 1.0);
        p0 = p1; p1 = p2;
    }
    *p = p1;
    /* P_n'(y) = n (y P_n - P_{n-1}) / (y^2 - 1) */
    *dp = n * (y * p1 - p0) / (y * y - 1.0);
}

/* n-point Gauss-Legendre rule on [0,1]: Newton's method on P_n(2 xi - 1),
 * started from the Chebyshev-like guess cos(pi (k + 3/4) / (n + 1/2)).
 * Weights 2/((1-y^2) P_n'(y)^2) on [-1,1], halved for [0,1]. */
int orc_gauss_legendre(int n, double *x, double *w)
{
    if (n < 1 || n > ORC_MAXN) return -1;
    for (int k = 0; k < n; ++k) {
        double y = cos(M_PI * (k + 0.75) / (n + 0.5));
        double p, dp;
        for (int it = 0; it < 100; ++it) {
            legendre(n, y, &p, &dp);
            double dy = p / dp;
            y -= dy;
            if (fabs(dy) < 1e-16) break;
        }
        legendre(n, y, &p, &dp);
        /* y runs from +1 downwards; store nodes in increasing order */
        x[n - 1 - k] = 0.5 * (y + 1.0);
        w[n - 1 - k] = 1.0 / ((1.0 - y * y) * dp * dp);
    }
    return 0;
}

/* Lagrange polynomials through the nodes, evaluated at xi:
 * phi_k(xi) = prod_{j != k} (xi - x_j) / (x_k - x_j). */
void orc_lagrange_eval(int n, const double *nodes, double xi, double *phi)
{
    for (int k = 0; k < n; ++k) {
        double v = 1.0;
        for (int j = 0; j < n; ++j)
            if (j != k) v *= (xi - nodes[j]) / (nodes[k] - nodes[j]);
        phi[k] = v;
    }
}

/* Derivative of each Lagrange polynomial at xi, by the product rule:
 * phi_k'(xi) = sum_{l != k} 1/(x_k - x_l) prod_{j != k,l} (xi - x_j)/(x_k - x_j). */
void orc_lagrange_deriv(int n, const double *nodes, double xi, double *dphi)
{
    for (int k = 0; k < n; ++k) {
        double s = 0.0;
        for (int l = 0; l < n; ++l) {
            if (l == k) continue;
            double prod = 1.0 / (nodes[k] - nodes[l]);
            for (int j = 0; j < n; ++j)
                if (j != k && j != l) prod *= (xi - nodes[j]) / (nodes[k] - nodes[j]);
            s += prod;
        }
        dphi[k] = s;
    }
}

/* The 1D operators of the scheme, row-major n x n:
 *   Dhat[j][k] = phi_k'(x_j)                 (nodal derivative, eq. D_kl times h)
 *   Kxi[k][l]  = int_0^1 phi_k'(xi) phi_l(xi) dxi   (volume / time stiffness)
 *   K1[k][l]   = phi_k(1) phi_l(1) - Kxi[k][l]      (eq. pde.st2 in time)
 *   F0[k] = phi_k(0), F1[k] = phi_k(1).
 * Kxi is computed with a separate (n+2)-point Gauss rule, i.e. from its
 * definition as an integral, not from Dhat. */
int orc_operators(int n, double *x, double *w, double *Dhat, double *Kxi,
                  double *K1, double *F0, double *F1)
{
    if (orc_gauss_legendre(n, x, w)) return -1;
    double phi[ORC_MAXN], dphi[ORC_MAXN];
    for (int j = 0; j < n; ++j) {
        orc_lagrange_deriv(n, x, x[j], dphi);
        for (int k = 0; k < n; ++k) Dhat[j * n + k] = dphi[k];
    }
    orc_lagrange_eval(n, x, 0.0, F0);
    orc_lagrange_eval(n, x, 1.0, F1);
    int nq = n + 2;
    double xq[ORC_MAXN + 2], wq[ORC_MAXN + 2];
    if (nq > ORC_MAXN) {
        /* n + 2 > table limit only for n > 8; fall back to n + 1 points,
         * still exact for the degree 2N - 1 integrand */
        nq = n + 1 <= ORC_MAXN ? n + 1 : n;
    }
    orc_gauss_legendre(nq, xq, wq);
    for (int k = 0; k < n * n; ++k) Kxi[k] = 0.0;
    for (int q = 0; q < nq; ++q) {
        orc_lagrange_eval(n, x, xq[q], phi);
        orc_lagrange_deriv(n, x, xq[q], dphi);
        for (int k = 0; k < n; ++k)
            for (int l = 0; l < n; ++l)
                Kxi[k * n + l] += wq[q] * dphi[k] * phi[l];
    }
    for (int k = 0; k < n; ++k)
        for (int l = 0; l < n; ++l)
            K1[k * n + l] = F1[k] * F1[l] - Kxi[k * n + l];
    return 0;
}

/* ------------------------------------------------------------------------ */
/* PDE functions: flux F_d(Q) and max |eigenvalue| of A.n for n = e_d        */
/* ------------------------------------------------------------------------ */

int orc_nvar(int pde, int dim)
{
    if (pde == 1) return 1;
    if (pde == 2) return dim + 2;
    if (pde == 3) return 9;
    if (pde == 4) return dim == 3 ? 13 : (dim == 2 ? 9 : -1);
    return -1;
}

/* Evolved variables: the leading ones.  The diffuse-interface system's last
 * four (alpha, lambda, mu, rho) obey q_t = 0. */
int orc_nevolved(const orc_cfg *c) { return c->pde == 4 ? c->m - 4 : c->m; }

/* Sec. 3.1 eq. euler, ideal gas p = (gamma-1)(rhoE - rho|v|^2/2). */
static void euler_flux(int dim, double gamma, const double *q, int d, double *f)
{
    double rho = q[0];
    double v[3] = {0.0, 0.0, 0.0};
    double kin = 0.0;
    for (int k = 0; k < dim; ++k) { v[k] = q[1 + k] / rho; kin += q[1 + k] * v[k]; }
    double E = q[dim + 1];
    double p = (gamma - 1.0) * (E - 0.5 * kin);
    f[0] = q[1 + d];
    for (int k = 0; k < dim; ++k) f[1 + k] = q[1 + k] * v[d] + (k == d ? p : 0.0);
    f[dim + 1] = v[d] * (E + p);
}

static double euler_eig(int dim, double gamma, const double *q, int d)
{
    double rho = q[0];
    double kin = 0.0;
    for (int k = 0; k < dim; ++k) kin += q[1 + k] * q[1 + k] / rho;
    double p = (gamma - 1.0) * (q[dim + 1] - 0.5 * kin);
    double c = sqrt(gamma * p / rho);
    return fabs(q[1 + d] / rho) + c;
}

/* Velocity-stress elasticity, Q = (sxx, syy, szz, sxy, syz, sxz, u, v, w):
 * sigma_t - E(lambda,mu) : grad v = 0,  rho v_t - div sigma = 0
 * (Sec. 3.2 with alpha = 1), written as Q_t + div F = 0. */
static void elastic_flux(const double *prm, const double *q, int d, double *f)
{
    double rho = prm[0], lam = prm[1], mu = prm[2];
    double sxx = q[0], syy = q[1], szz = q[2], sxy = q[3], syz = q[4], sxz = q[5];
    double u = q[6], v = q[7], w = q[8];
    (void)syy; (void)szz;
    double vel[3] = {u, v, w};
    /* normal stress rows: -(lambda + 2 mu delta_{ii,d}) v_d */
    for (int i = 0; i < 3; ++i) f[i] = -(lam + (i == d ? 2.0 * mu : 0.0)) * vel[d];
    /* shear rows: sxy couples (x,y), syz (y,z), sxz (x,z) */
    f[3] = d == 0 ? -mu * v : (d == 1 ? -mu * u : 0.0);
    f[4] = d == 1 ? -mu * w : (d == 2 ? -mu * v : 0.0);
    f[5] = d == 0 ? -mu * w : (d == 2 ? -mu * u : 0.0);
    /* momentum rows: -(sigma . e_d) / rho */
    double s_row[3][3] = {{sxx, sxy, sxz}, {sxy, q[1], syz}, {sxz, syz, q[2]}};
    for (int i = 0; i < 3; ++i) f[6 + i] = -s_row[i][d] / rho;
}

/* Diffuse-interface linear elasticity (Sec. 3.2), reading R19:
 *   sigma_t - E : (1/alpha) grad(alpha v) + (1/alpha) E : (v (x) grad alpha) = 0
 *   (alpha v)_t - (alpha/rho) div sigma - (1/rho) sigma grad alpha = 0
 *   alpha_t = lambda_t = mu_t = rho_t = 0
 * with E : G = lambda tr(G) I + mu (G + G^T) (Hooke's law on the velocity
 * gradient) and state Q = (sigma, w = alpha v, alpha, lambda, mu, rho),
 * sigma in the order xx yy zz xy yz xz (3D) or xx yy xy (2D).  There is no
 * flux; every term is a non-conservative product B_d(Q) dQ/dx_d:
 *   a_i = (1/alpha) dw_i/dx_d - (w_i/alpha^2) dalpha/dx_d   (= dv_i/dx_d)
 *   sigma_ij row: -(lambda a_d delta_ij + mu (a_i delta_jd + delta_id a_j))
 *   w_i row:      -(alpha dsigma_id/dx_d + sigma_id dalpha/dx_d) / rho
 * nc_out = B_d(q) g for the derivative vector g = dQ/dx_d. */
static int sym_index(int dim, int i, int j)
{
    if (i > j) { int t = i; i = j; j = t; }
    if (dim == 2) return i == j ? i : 2;
    if (i == j) return i;
    return (i == 0 && j == 1) ? 3 : ((i == 1 && j == 2) ? 4 : 5);
}

static void dim_ncp(int dim, const double *q, int d, const double *g, double *out)
{
    const int nsig = dim == 3 ? 6 : 3;
    const double *w = q + nsig;
    const double alpha = q[nsig + dim], lam = q[nsig + dim + 1], mu = q[nsig + dim + 2], rho = q[nsig + dim + 3];
    const double ga = g[nsig + dim];
    double a[3];
    for (int i = 0; i < dim; ++i) a[i] = g[nsig + i] / alpha - w[i] * ga / (alpha * alpha);
    for (int i = 0; i < dim; ++i)
        for (int j = i; j < dim; ++j) {
            double r = -mu * ((j == d ? a[i] : 0.0) + (i == d ? a[j] : 0.0));
            if (i == j) r -= lam * a[d];
            out[sym_index(dim, i, j)] = r;
        }
    for (int i = 0; i < dim; ++i) {
        const int k = sym_index(dim, i, d);
        out[nsig + i] = -(alpha * g[k] + q[k] * ga) / rho;
    }
    for (int v = nsig + dim; v < nsig + dim + 4; ++v) out[v] = 0.0;
}

void orc_flux(const orc_cfg *c, const double *q, int d, double *f)
{
    if (c->pde == 1) f[0] = c->prm[d] * q[0];
    else if (c->pde == 2) euler_flux(c->dim, c->prm[0], q, d, f);
    else if (c->pde == 3) elastic_flux(c->prm, q, d, f);
    else for (int v = 0; v < c->m; ++v) f[v] = 0.0;
}

/* Non-conservative product B_d(q) g (eq. pde); zero for the conservative
 * systems. */
void orc_ncp(const orc_cfg *c, const double *q, int d, const double *g, double *out)
{
    if (c->pde == 4) dim_ncp(c->dim, q, d, g, out);
    else for (int v = 0; v < c->m; ++v) out[v] = 0.0;
}

/* Algebraic source S(q) (eq. pde): -kappa q for advection, zero otherwise. */
void orc_source(const orc_cfg *c, const double *q, double *S)
{
    for (int v = 0; v < c->m; ++v) S[v] = c->pde == 1 ? -c->prm[3] * q[v] : 0.0;
}

double orc_max_eig(const orc_cfg *c, const double *q, int d)
{
    if (c->pde == 1) return fabs(c->prm[d]);
    if (c->pde == 2) return euler_eig(c->dim, c->prm[0], q, d);
    if (c->pde == 3) return sqrt((c->prm[1] + 2.0 * c->prm[2]) / c->prm[0]);
    /* diffuse interface: the P-wave speed; the eigenvalues do not depend on
     * alpha (Sec. 3.2) */
    const int b = c->m - 3;
    return sqrt((q[b] + 2.0 * q[b + 1]) / q[b + 2]);
}

/* ------------------------------------------------------------------------ */
/* Helpers                                                                   */
/* ------------------------------------------------------------------------ */

static int ipow(int b, int e) { int r = 1; while (e-- > 0) r *= b; return r; }

static double cell_dx(const orc_cfg *c, int d)
{
    return (c->hi[d] - c->lo[d]) / c->cells[d];
}

/* digit k of the base-n multi-index s */
static int digit(int s, int n, int k) { for (int i = 0; i < k; ++i) s /= n; return s % n; }

/* s with its digit k replaced by j */
static int with_digit(int s, int n, int k, int j)
{
    int p = ipow(n, k);
    return s - digit(s, n, k) * p + j * p;
}

/* face index of s on a face normal to d: the other digits in increasing order */
static int face_index(int s, int n, int dim, int d)
{
    int p = 0, mul = 1;
    for (int k = 0; k < dim; ++k) {
        if (k == d) continue;
        p += digit(s, n, k) * mul;
        mul *= n;
    }
    return p;
}

/* LU factorisation with partial pivoting (Doolittle), in place. */
static int lu_factor(int n, double *A, int *piv)
{
    for (int k = 0; k < n; ++k) {
        int p = k;
        for (int i = k + 1; i < n; ++i) if (fabs(A[i * n + k]) > fabs(A[p * n + k])) p = i;
        if (A[p * n + k] == 0.0) return -1;
        piv[k] = p;
        if (p != k) for (int j = 0; j < n; ++j) { double t = A[k * n + j]; A[k * n + j] = A[p * n + j]; A[p * n + j] = t; }
        for (int i = k + 1; i < n; ++i) {
            A[i * n + k] /= A[k * n + k];
            for (int j = k + 1; j < n; ++j) A[i * n + j] -= A[i * n + k] * A[k * n + j];
        }
    }
    return 0;
}

static void lu_solve(int n, const double *LU, const int *piv, double *b)
{
    for (int k = 0; k < n; ++k) if (piv[k] != k) { double t = b[k]; b[k] = b[piv[k]]; b[piv[k]] = t; }
    for (int i = 1; i < n; ++i) for (int j = 0; j < i; ++j) b[i] -= LU[i * n + j] * b[j];
    for (int i = n - 1; i >= 0; --i) {
        for (int j = i + 1; j < n; ++j) b[i] -= LU[i * n + j] * b[j];
        b[i] /= LU[i * n + i];
    }
}

typedef struct {
    int n;
    double x[ORC_MAXN], w[ORC_MAXN], F0[ORC_MAXN], F1[ORC_MAXN];
    double Dhat[ORC_MAXN * ORC_MAXN], Kxi[ORC_MAXN * ORC_MAXN], K1[ORC_MAXN * ORC_MAXN];
    double K1lu[ORC_MAXN * ORC_MAXN];
    int piv[ORC_MAXN];
} basis;

static int make_basis(int N, basis *b)
{
    b->n = N + 1;
    if (orc_operators(b->n, b->x, b->w, b->Dhat, b->Kxi, b->K1, b->F0, b->F1)) return -1;
    memcpy(b->K1lu, b->K1, sizeof(b->K1));
    return lu_factor(b->n, b->K1lu, b->piv);
}

/* Default Picard count: N+1 from the trivial guess (reading R3); an
 * initial guess of degree k in time (k = 1, 2 for guesses 1, 2) is already
 * of order k+1, so one iteration fewer per degree: N+1-k, at least 1.  The
 * paper's sufficiency rule (a degree N-1 guess needs one iteration, Sec.
 * 2.2) corresponds to N-k; the default keeps the one extra iteration the
 * trivial guess has. */
static int cerk_order(int N);

int orc_picard_count(const orc_cfg *c)
{
    if (c->picard != 0) return c->picard;
    if (c->guess == 3) return 2;  /* a degree-N guess: one iteration, plus one */
    int P = c->N + 1 - (c->guess == 1 ? 1 : c->guess == 2 ? 2 : c->guess == 4 ? cerk_order(c->N) : 0);
    return P < 1 ? 1 : P;
}

/* Picard count of a step of the extrapolation guess that has no previous
 * predictor (it takes the third-order guess and its default count). */
static int fallback_picard(const orc_cfg *c)
{
    int P = c->N + 1 - 2;
    return P < 1 ? 1 : P;
}

/* Default CFL coefficient alpha(N) = 0.9 x the von Neumann stability limit
 * of this scheme for 1D linear advection (the paper's bound alpha < 1/(2N+1)
 * of Sec. 3 is necessary, not sufficient; it defers the actual limit to a
 * von Neumann analysis).  The limits 0.3335, 0.1709, 0.1040, 0.0699, 0.0501,
 * 0.0377, 0.0294, 0.0236, 0.0193 (N = 1..9) are recomputed from this
 * oracle's own step operator by the stability test. */
static const double alpha_default[10] = {
    0.9, 0.3001, 0.1538, 0.0936, 0.0629, 0.0451, 0.0339, 0.0265, 0.0212, 0.0174};

double orc_alpha(const orc_cfg *c)
{
    if (c->alpha > 0.0) return c->alpha;
    return (c->N >= 0 && c->N <= 9) ? alpha_default[c->N] : 0.5 / (2.0 * c->N + 1.0);
}

/* ------------------------------------------------------------------------ */
/* Space-time predictor (Sec. 2.2, eq. pde.st2) for one element              */
/* ------------------------------------------------------------------------ */

/* In nodal form, with diagonal mass and GL quadrature, eq. pde.st2 divided by
 * |Omega| w_s reads, for every spatial node s and variable v,
 *     sum_l K1[t][l] q[l][s] = F0[t] u[s] + dt w_t R[t][s],
 *     R[t][s] = - sum_d (1/dx_d) sum_j Dhat[s_d][j] F_d(q[t][s|d=j]).
 * Picard: evaluate R at the previous iterate, solve the n x n time system.
 *
 * Outputs (any may be NULL): qhat[t][s][v] (n^{d+1} m), qbar[s][v] (n^d m),
 * Fbar[d][s][v] (dim n^d m).  Returns the number of iterations done. */
/* L(w) = S(w) - sum_d (1/dx_d) [Dhat_d F_d(w) + B_d(w) Dhat_d w] at the
 * spatial nodes of one element: the element-local approximation of the time
 * derivative of Sec. 2.2 (the L operator), with the same nodal derivative as
 * the predictor (reading R2); with_flux = 0 leaves out the flux divergence
 * (the corrector's volume integrals of B and S).  tmp holds dim ns m values. */
static void l_eval(const orc_cfg *c, const basis *b, const double *w, double *Lw, double *tmp, int with_flux)
{
    const int n = b->n, dim = c->dim, m = c->m, ns = ipow(n, dim);
    if (with_flux)
        for (int d = 0; d < dim; ++d)
            for (int s = 0; s < ns; ++s) orc_flux(c, &w[(size_t)s * m], d, &tmp[((size_t)d * ns + s) * m]);
    for (int s = 0; s < ns; ++s) {
        double r[ORC_MAXM];
        orc_source(c, &w[(size_t)s * m], r);
        for (int d = 0; d < dim; ++d) {
            const int sd = digit(s, n, d);
            double g[ORC_MAXM], nc[ORC_MAXM];
            for (int v = 0; v < m; ++v) {
                double acc = 0.0, ga = 0.0;
                for (int j = 0; j < n; ++j) {
                    const int sj = with_digit(s, n, d, j);
                    if (with_flux) acc += b->Dhat[sd * n + j] * tmp[((size_t)d * ns + sj) * m + v];
                    ga += b->Dhat[sd * n + j] * w[(size_t)sj * m + v];
                }
                if (with_flux) r[v] -= acc / cell_dx(c, d);
                g[v] = ga;
            }
            orc_ncp(c, &w[(size_t)s * m], d, g, nc);
            for (int v = 0; v < m; ++v) r[v] -= nc[v] / cell_dx(c, d);
        }
        for (int v = 0; v < m; ++v) Lw[(size_t)s * m + v] = r[v];
    }
}

static void l_operator(const orc_cfg *c, const basis *b, const double *w, double *Lw, double *tmp)
{
    l_eval(c, b, w, Lw, tmp, 1);
}

/* The PDE has a non-conservative product or a source (a volume integral
 * beyond the flux term). */
static int has_nc_or_source(const orc_cfg *c) { return c->pde == 4 || (c->pde == 1 && c->prm[3] != 0.0); }

/* Continuous explicit Runge-Kutta (CERK) schemes for the CERK guess
 * (Sec. 2.2 names the continuous extensions of Owren and Zennaro and prints
 * no coefficients).  A scheme of s stages takes k_i = L(u + dt sum_{j<i}
 * a_ij k_j) and has the dense output u(t^n + th dt) ~ u + dt sum_i b_i(th)
 * k_i with polynomial weights b_i(th) = sum_k beta_ik th^(k+1) (no constant
 * term).  It has uniform order p when, for every rooted tree t of order
 * |t| <= p with elementary weights Phi_i(t) and density gamma(t),
 *   sum_i b_i(th) Phi_i(t) = th^|t| / gamma(t)   for every th in [0, 1],
 * so the dense output is a polynomial of degree p in time whose error is
 * O(dt^(p+1)) uniformly in th.
 *   order 3: the classical fourth-order method (stages at 0, 1/2, 1/2, 1,
 *     a21 = a32 = 1/2, a43 = 1) with the cubic dense output that ends in its
 *     weights 1/6, 1/3, 1/3, 1/6 at th = 1:
 *     b1 = th - 3 th^2/2 + 2 th^3/3, b2 = b3 = th^2 - 2 th^3/3,
 *     b4 = -th^2/2 + 2 th^3/3;
 *   order 4: six stages with quartic weights.  Five stages do not reach
 *     uniform order 4; this six-stage tableau was found by a numerical
 *     search over the stage coefficients, minimising max |b_i(th)| on
 *     [0, 1] (0.35) with nodes c_i in [0, 1], then solved to 40 digits by
 *     Newton's method on the eight order conditions;
 *   order 5: eleven stages with quintic weights, found the same way (the
 *     seventeen conditions of the trees of order <= 5, the weights
 *     eliminated by least squares, a penalty on |b_i(th)| and |a_ij|):
 *     max |b_i(th)| 0.31, max |a_ij| 0.48, nodes c_i in [0, 0.88].
 * The values below are those digits rounded to 20; the order conditions
 * hold to rounding (pinned in the tests). */
#define ORC_CERK_SMAX 11
typedef struct {
    int s, p;
    double a[ORC_CERK_SMAX][ORC_CERK_SMAX];
    double beta[ORC_CERK_SMAX][6];
} cerk_scheme;

static const cerk_scheme cerk_order3 = {
    4, 3,
    {{0}, {0.5}, {0.0, 0.5}, {0.0, 0.0, 1.0}},
    {{1.0, -1.5, 2.0 / 3.0}, {0.0, 1.0, -2.0 / 3.0}, {0.0, 1.0, -2.0 / 3.0}, {0.0, -0.5, 2.0 / 3.0}},
};

static const cerk_scheme cerk_order4 = {
    6, 4,
    {{0},
     {0.50849583384840113958},
     {0.046949965621769603951, 0.4819237260551746206},
     {0.16975684152901151769, 0.071063883183927482688, -0.028300707574148454932},
     {-0.076143308578057834897, -0.14017373747662979618, 0.048722116369755792049, 0.50735746259681266958},
     {0.12216705712724082426, 0.12299809408491295783, 0.48070156394276517752, 0.02616528026761548546,
      0.093926602975396757805}},
    {{1.0, -3.9153671327673924417, 5.9934951934142588637, -3.0269093126242169958},
     {0.0, -0.80100882679982742762, 2.6530980786357989255, -1.7516658795402877462},
     {0.0, -0.89842534403733875434, 2.9131919603555952085, -1.8758298804924840825},
     {0.0, 5.3725609369242888065, -13.195842800637089784, 8.1610686740032049053},
     {0.0, -0.070646768460630971334, 2.90293867489981116, -2.8111171676340170791},
     {0.0, 0.31288713514090078845, -1.2668811066683743739, 1.3044535662878009984}},
};

static const cerk_scheme cerk_order5 = {
    11, 5,
    {{0},
     {0.21396406893114929941},
     {0.034520790017671977007, 0.41372592912176714349},
     {0.088416642665365227537, 0.13683623308249277562, 0.47755326751379046974},
     {-0.0266719632876990541, 0.12845891088304249121, 0.073770359528602792921, -0.029901862330888622484},
     {0.15811896403112403656, 0.062824176896518388083, -0.040310351902863277689, -0.19180775673017479455,
      0.093904496963942459173},
     {0.095444096258275612407, 0.029612493702906972604, 0.042065059631820178293, 0.056639453843974274155,
      0.23157141256193104679, -0.082321405762062763284},
     {-0.0099858386067894141076, -0.004311214382797107593, 0.042484710026669023005, -0.061702579717549094049,
      0.1360902187699344359, 0.089703158714395027355, 0.093344465039202374441},
     {0.044225647283319301368, 0.038507705255559191753, -0.12347160217482120146, 0.013995747001842868748,
      0.091397903235836837048, 0.017790975806619039112, 0.022029539570705958954, -0.0069441602114276107782},
     {0.040551492362699865282, 0.12072433771358202958, 0.042059965202631322386, 0.36018691033467310849,
      0.038926340292962444834, -0.0061070210341534810037, 0.16681162009247751788, 0.019144269354406344107,
      0.08877318014754002403},
     {0.080638694974360216797, 0.01205941886818835392, 0.018096630449363849, 0.055867998305249973877,
      0.091187420805903382723, -0.0089338243342328581078, 0.24597832827170908575, 0.04717166509034146719,
      0.048963914391693246618, 0.021076563758733234774}},
    {{1.0, -6.6143117173026234553, 17.178359569284717945, -18.86793234430243545, 7.3659907185475543609},
     {0.0, 2.1719103255203805044, -7.2952295061885010417, 8.9606564533760370553, -3.8193824401789661292},
     {0.0, -1.5854789298302827005, 9.4423133346087880382, -15.145534664537743023, 7.4773099169377650253},
     {0.0, 0.88423518048995741019, -5.35768986153765167, 10.111281515466986061, -5.6462993048931384541},
     {0.0, 3.2971257036516648115, -12.513611374370090692, 16.088923484236408098, -6.8449476884926829149},
     {0.0, -0.31163502670566630635, 1.0070308771872418124, -1.1615838865360656713, 0.45679117132443454501},
     {0.0, -0.78236688921344789434, 6.1477951147591089282, -10.406910275786306437, 5.1537555111704861162},
     {0.0, -1.5146597261084853013, 8.8458108856981437369, -13.086412777562555403, 5.8623322128438347029},
     {0.0, 4.3645676908433573827, -15.732556849961202994, 19.346795749644294217, -7.8916086488488356334},
     {0.0, -0.33452411430651430281, 2.3248704578988559346, -5.0045221963152205875, 3.3202049045619430229},
     {0.0, 0.42513750296165985198, -4.0470926473794099978, 9.1652389423166011406, -5.4341463529723946416}},
};

/* The scheme of the CERK guess for degree N: the paper's rule wants a guess
 * of degree N - 1 in time (one Picard iteration then suffices), so order
 * N - 1, at least 3 and at most the highest order built (5). */
static const cerk_scheme *cerk_for(int N)
{
    return N >= 6 ? &cerk_order5 : N >= 5 ? &cerk_order4 : &cerk_order3;
}

static int cerk_order(int N) { return cerk_for(N)->p; }

/* Tableau of the CERK guess for degree N: a[i * s + j] (row-major s x s,
 * zero on and above the diagonal) and beta[i * p + k] (b_i(th) = sum_k
 * beta_ik th^(k+1)).  Returns s; *p receives the order. */
int orc_cerk_scheme(int N, double *a, double *beta, int *p)
{
    const cerk_scheme *cs = cerk_for(N);
    for (int i = 0; i < cs->s; ++i) {
        for (int j = 0; j < cs->s; ++j) a[i * cs->s + j] = j < i ? cs->a[i][j] : 0.0;
        for (int k = 0; k < cs->p; ++k) beta[i * cs->p + k] = cs->beta[i][k];
    }
    *p = cs->p;
    return cs->s;
}

/* b_i(th) of the CERK guess for degree N (s values). */
void orc_cerk_weights(int N, double th, double *bw)
{
    const cerk_scheme *cs = cerk_for(N);
    for (int i = 0; i < cs->s; ++i) {
        double v = 0.0, thk = th;
        for (int k = 0; k < cs->p; ++k) {
            v += cs->beta[i][k] * thk;
            thk *= th;
        }
        bw[i] = v;
    }
}

/* Initial guess q0 at the space-time nodes (t^n + tau_t, x_s),
 * tau_t = xi_t dt (Sec. 2.2, written as a Taylor series in time):
 *   0: q0 = u (the trivial guess)
 *   1: q0 = u + tau L(u)                                  (second order)
 *   2: q0 = u + tau k1 + tau^2 (k2 - k1) / (2 dt),
 *      k1 = L(u), k2 = L(u + dt k1)                       (third order)
 *   3: the previous step's predictor qprev (n time nodes on its interval of
 *      length dt / ratio) extrapolated in time past its end and shifted to
 *      start at u:  q0 = u + qprev(1 + xi_t ratio) - qprev(1), the
 *      polynomials evaluated with the Lagrange basis of the time nodes;
 *      without qprev, guess 2.
 *   4: the CERK guess (Sec. 2.2 names continuous extension Runge-Kutta
 *      schemes): k_i = L(u + dt sum_{j<i} a_ij k_j), q0 = u + dt sum_i
 *      b_i(tau/dt) k_i with the scheme of order min(5, max(3, N - 1))
 *      (cerk_for)
 * gw holds guess_work_len(c) values. */
static size_t guess_work_len(const orc_cfg *c)
{
    return (size_t)ipow(c->N + 1, c->dim) * c->m * (ORC_CERK_SMAX + 1 + c->dim);
}

static void initial_guess(const orc_cfg *c, const basis *b, const double *u, double dt, double *q,
                          double *gw, const double *qprev, double ratio)
{
    const int n = b->n, ns = ipow(n, c->dim), m = c->m;
    const size_t nsm = (size_t)ns * m;
    if (c->guess == 3 && qprev) {
        double L1[ORC_MAXN];
        orc_lagrange_eval(n, b->x, 1.0, L1);
        for (int t = 0; t < n; ++t) {
            double Lt[ORC_MAXN];
            orc_lagrange_eval(n, b->x, 1.0 + b->x[t] * ratio, Lt);
            for (size_t i = 0; i < nsm; ++i) {
                double v = u[i];
                for (int k = 0; k < n; ++k) v += (Lt[k] - L1[k]) * qprev[(size_t)k * nsm + i];
                q[(size_t)t * nsm + i] = v;
            }
        }
        return;
    }
    if (c->guess == 4) {
        const cerk_scheme *cs = cerk_for(c->N);
        double *k = gw, *w = gw + (size_t)ORC_CERK_SMAX * nsm, *tmp = w + nsm;  /* k_i at k + i nsm */
        for (int st = 0; st < cs->s; ++st) {
            for (size_t i = 0; i < nsm; ++i) {
                double acc = 0.0;
                for (int j = 0; j < st; ++j) acc += cs->a[st][j] * k[(size_t)j * nsm + i];
                w[i] = u[i] + dt * acc;
            }
            l_operator(c, b, w, k + (size_t)st * nsm, tmp);
        }
        for (int t = 0; t < n; ++t) {
            double bw[ORC_CERK_SMAX];
            orc_cerk_weights(c->N, b->x[t], bw);
            for (size_t i = 0; i < nsm; ++i) {
                double acc = 0.0;
                for (int st = 0; st < cs->s; ++st) acc += bw[st] * k[(size_t)st * nsm + i];
                q[(size_t)t * nsm + i] = u[i] + dt * acc;
            }
        }
        return;
    }
    const int g = c->guess == 3 ? 2 : c->guess;
    double *k1 = gw, *k2 = gw + nsm, *w = gw + 2 * nsm, *tmp = gw + 3 * nsm;
    if (g == 1 || g == 2) l_operator(c, b, u, k1, tmp);
    if (g == 2) {
        for (size_t i = 0; i < nsm; ++i) w[i] = u[i] + dt * k1[i];
        l_operator(c, b, w, k2, tmp);
    }
    for (int t = 0; t < n; ++t) {
        const double tau = b->x[t] * dt;
        for (size_t i = 0; i < nsm; ++i) {
            double v = u[i];
            if (g == 1 || g == 2) v += tau * k1[i];
            if (g == 2) v += 0.5 * tau * tau * (k2[i] - k1[i]) / dt;
            q[(size_t)t * nsm + i] = v;
        }
    }
}

static int predictor_elem(const orc_cfg *c, const basis *b, const double *u, double dt,
                          double *qhat, double *qbar, double *Fbar, double *work,
                          const double *qprev, double ratio)
{
    const int n = b->n, dim = c->dim, m = c->m;
    const int ns = ipow(n, dim), nst = n * ns;
    double *q = work;                     /* nst m */
    double *F = q + (size_t)nst * m;      /* dim nst m */
    double *R = F + (size_t)dim * nst * m;/* nst m */
    double *qn = R + (size_t)nst * m;     /* nst m */
    initial_guess(c, b, u, dt, q, work + (size_t)nst * m * (3 + dim), qprev, ratio);

    int P = (c->guess == 3 && !qprev) ? fallback_picard(c) : orc_picard_count(c);
    int to_conv = P < 0;
    int maxit = to_conv ? 50 : P;
    int it;
    for (it = 0; it < maxit; ++it) {
        /* R = L(q) at every time node: S - sum_d (Dhat_d F_d + B_d Dhat_d q) / dx_d */
        for (int t = 0; t < n; ++t) l_eval(c, b, &q[(size_t)t * ns * m], &R[(size_t)t * ns * m], F, 1);
        double dmax = 0.0, qmax = 0.0;
        for (int s = 0; s < ns; ++s)
            for (int v = 0; v < m; ++v) {
                double rhs[ORC_MAXN];
                for (int t = 0; t < n; ++t)
                    rhs[t] = b->F0[t] * u[(size_t)s * m + v] + dt * b->w[t] * R[((size_t)t * ns + s) * m + v];
                lu_solve(n, b->K1lu, b->piv, rhs);
                for (int t = 0; t < n; ++t) {
                    size_t idx = ((size_t)t * ns + s) * m + v;
                    double dq = fabs(rhs[t] - q[idx]);
                    if (dq > dmax) dmax = dq;
                    if (fabs(rhs[t]) > qmax) qmax = fabs(rhs[t]);
                    qn[idx] = rhs[t];
                }
            }
        memcpy(q, qn, sizeof(double) * (size_t)nst * m);
        if (to_conv && dmax <= 1e-14 * qmax) { ++it; break; }
    }

    /* time averages: qbar = sum_t w_t q[t], Fbar_d = sum_t w_t F_d(q[t]) */
    for (int d = 0; d < dim; ++d)
        for (int l = 0; l < nst; ++l)
            orc_flux(c, &q[(size_t)l * m], d, &F[((size_t)d * nst + l) * m]);
    if (qhat) memcpy(qhat, q, sizeof(double) * (size_t)nst * m);
    if (qbar)
        for (int s = 0; s < ns; ++s)
            for (int v = 0; v < m; ++v) {
                double acc = 0.0;
                for (int t = 0; t < n; ++t) acc += b->w[t] * q[((size_t)t * ns + s) * m + v];
                qbar[(size_t)s * m + v] = acc;
            }
    if (Fbar)
        for (int d = 0; d < dim; ++d)
            for (int s = 0; s < ns; ++s)
                for (int v = 0; v < m; ++v) {
                    double acc = 0.0;
                    for (int t = 0; t < n; ++t) acc += b->w[t] * F[((size_t)d * nst + (size_t)t * ns + s) * m + v];
                    Fbar[((size_t)d * ns + s) * m + v] = acc;
                }
    return it;
}

static size_t predictor_work_len(const orc_cfg *c)
{
    int n = c->N + 1;
    size_t nst = (size_t)ipow(n, c->dim + 1), ns = (size_t)ipow(n, c->dim);
    (void)ns;
    return nst * c->m * (3 + c->dim) + guess_work_len(c);
}

/* Volume integral of the corrector (third integral of eq. pde.nc.gw2) divided
 * by the diagonal mass |Omega| w_s and by dt:
 *   V[s][v] = sum_d (1/dx_d)(1/w_{s_d}) sum_j Kxi[s_d][j] Fbar_d[s|d=j][v]. */
static void volume_elem(const orc_cfg *c, const basis *b, const double *Fbar, double *V)
{
    const int n = b->n, dim = c->dim, m = c->m, ns = ipow(n, dim);
    for (int s = 0; s < ns; ++s)
        for (int v = 0; v < m; ++v) {
            double acc = 0.0;
            for (int d = 0; d < dim; ++d) {
                int sd = digit(s, n, d);
                double a = 0.0;
                for (int j = 0; j < n; ++j)
                    a += b->Kxi[sd * n + j] * Fbar[((size_t)d * ns + with_digit(s, n, d, j)) * m + v];
                acc += a / (cell_dx(c, d) * b->w[sd]);
            }
            V[(size_t)s * m + v] = acc;
        }
}

/* Volume integrals of the non-conservative product and the source (fourth
 * and fifth integrals of eq. pde.nc.gw2), divided by the diagonal mass and
 * by dt, added to V: with the nodal quadrature in space and the time nodes
 * in time, V[s] += sum_t w_t [S(q_t) - sum_d (1/dx_d) B_d(q_t) Dhat_d q_t](x_s).
 * qhat[t][s][v] is the predictor; tmp holds 2 ns m values. */
static void volume_nc_elem(const orc_cfg *c, const basis *b, const double *qhat, double *V, double *tmp)
{
    const int n = b->n, m = c->m, ns = ipow(n, c->dim);
    double *Lt = tmp;
    for (int t = 0; t < n; ++t) {
        l_eval(c, b, &qhat[(size_t)t * ns * m], Lt, NULL, 0);
        for (size_t i = 0; i < (size_t)ns * m; ++i) V[i] += b->w[t] * Lt[i];
    }
}

/* Boundary extrapolation of the time averages to the 2d faces:
 *   qf[d][side][p][v] = sum_j phi_j(side) qbar[s(d=j,perp=p)][v]
 *   ff[d][side][p][v] = sum_j phi_j(side) Fbar_d[s(d=j,perp=p)][v]. */
static void traces_elem(const orc_cfg *c, const basis *b, const double *qbar, const double *Fbar,
                        double *qf, double *ff)
{
    const int n = b->n, dim = c->dim, m = c->m, ns = ipow(n, dim), nf = ipow(n, dim - 1);
    for (int d = 0; d < dim; ++d)
        for (int side = 0; side < 2; ++side) {
            const double *phi = side ? b->F1 : b->F0;
            for (int p = 0; p < nf; ++p)
                for (int v = 0; v < m; ++v) {
                    double aq = 0.0, af = 0.0;
                    for (int s = 0; s < ns; ++s) {
                        if (face_index(s, n, dim, d) != p) continue;
                        int j = digit(s, n, d);
                        aq += phi[j] * qbar[(size_t)s * m + v];
                        af += phi[j] * Fbar[((size_t)d * ns + s) * m + v];
                    }
                    size_t o = (((size_t)d * 2 + side) * nf + p) * m + v;
                    qf[o] = aq;
                    ff[o] = af;
                }
        }
}

/* Rusanov flux (eq. pc.scheme with B = 0, eq. rusanov), L = lower element,
 * R = upper element along d:
 *   F* = (fL + fR)/2 - s_max (qR - qL)/2, s_max = max(|lambda_d(qL)|, |lambda_d(qR)|). */
void orc_rusanov(const orc_cfg *c, int d, const double *qL, const double *fL,
                 const double *qR, const double *fR, double *fs)
{
    double sL = orc_max_eig(c, qL, d), sR = orc_max_eig(c, qR, d);
    double smax = sL > sR ? sL : sR;
    for (int v = 0; v < c->m; ++v) fs[v] = 0.5 * (fL[v] + fR[v]) - 0.5 * smax * (qR[v] - qL[v]);
}

/* Path integral of eq. pc.scheme along the straight segment
 * psi(s) = qL + s (qR - qL):  J = int_0^1 B_d(psi(s)) ds (qR - qL), by the
 * three-point Gauss-Legendre rule on [0,1] (nodes 1/2 -+ sqrt(3/5)/2 and
 * 1/2, weights 5/18, 8/18, 5/18). */
void orc_path_jump(const orc_cfg *c, int d, const double *qL, const double *qR, double *J)
{
    const double r = 0.5 * sqrt(0.6);
    const double sg[3] = {0.5 - r, 0.5, 0.5 + r}, wg[3] = {5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0};
    const int m = c->m;
    double dq[ORC_MAXM], psi[ORC_MAXM], b[ORC_MAXM];
    for (int v = 0; v < m; ++v) { dq[v] = qR[v] - qL[v]; J[v] = 0.0; }
    for (int k = 0; k < 3; ++k) {
        for (int v = 0; v < m; ++v) psi[v] = qL[v] + sg[k] * dq[v];
        orc_ncp(c, psi, d, dq, b);
        for (int v = 0; v < m; ++v) J[v] += wg[k] * b[v];
    }
}

/* Face fluctuations along d between the lower element (its xi_d = 1 trace
 * qL, fL) and the upper one (its xi_d = 0 trace qR, fR), each in the e_d
 * convention of the lift (eq. pc.scheme, eq. rusanov; readings R20, R21):
 *   f_lower = (fL + fR)/2 - Theta (qR - qL)/2 + J/2
 *   f_upper = (fL + fR)/2 - Theta (qR - qL)/2 - J/2
 * Theta = s_max on the evolved variables, 0 on the material parameters. */
void orc_face_flux(const orc_cfg *c, int d, const double *qL, const double *fL, const double *qR,
                   const double *fR, double *f_lower, double *f_upper)
{
    double sL = orc_max_eig(c, qL, d), sR = orc_max_eig(c, qR, d);
    double smax = sL > sR ? sL : sR;
    const int mev = orc_nevolved(c);
    double J[ORC_MAXM];
    orc_path_jump(c, d, qL, qR, J);
    for (int v = 0; v < c->m; ++v) {
        double f = 0.5 * (fL[v] + fR[v]) - (v < mev ? 0.5 * smax * (qR[v] - qL[v]) : 0.0);
        f_lower[v] = f + 0.5 * J[v];
        f_upper[v] = f - 0.5 * J[v];
    }
}

/* ------------------------------------------------------------------------ */
/* Exported element-level entry points                                       */
/* ------------------------------------------------------------------------ */

int orc_predictor(const orc_cfg *c, const double *u, double dt, double *qhat,
                  double *qbar, double *Fbar, int *iters)
{
    basis b;
    if (make_basis(c->N, &b)) return -1;
    double *work = malloc(sizeof(double) * predictor_work_len(c));
    if (!work) return -2;
    int it = predictor_elem(c, &b, u, dt, qhat, qbar, Fbar, work, NULL, 1.0);
    free(work);
    if (iters) *iters = it;
    return 0;
}

/* The extrapolation guess alone for one element, from a previous predictor
 * qprev ([n][n^d][m]) over an interval dt / ratio. */
int orc_initial_guess_extrap(const orc_cfg *c, const double *u, double dt, const double *qprev, double ratio,
                             double *q0)
{
    basis b;
    if (c->guess != 3 || make_basis(c->N, &b)) return -1;
    initial_guess(c, &b, u, dt, q0, NULL, qprev, ratio);
    return 0;
}

/* The initial guess alone (no Picard iteration) for one element. */
int orc_initial_guess(const orc_cfg *c, const double *u, double dt, double *q0)
{
    basis b;
    if (make_basis(c->N, &b)) return -1;
    double *gw = malloc(sizeof(double) * guess_work_len(c));
    if (!gw) return -2;
    initial_guess(c, &b, u, dt, q0, gw, NULL, 1.0);
    free(gw);
    return 0;
}

int orc_volume(const orc_cfg *c, const double *Fbar, double *V)
{
    basis b;
    if (make_basis(c->N, &b)) return -1;
    volume_elem(c, &b, Fbar, V);
    return 0;
}

int orc_traces(const orc_cfg *c, const double *qbar, const double *Fbar, double *qf, double *ff)
{
    basis b;
    if (make_basis(c->N, &b)) return -1;
    traces_elem(c, &b, qbar, Fbar, qf, ff);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Subcell operators of the limiter (Sec. 2.3)                               */
/* ------------------------------------------------------------------------ */

/* 1D: S = 2N+1 equal subcells of [0,1].
 *   Pr[j][k] = average of phi_k over subcell j (n-point GL per subcell:
 *              exact, the integrand has degree N)
 *   Rc[k][j] = least-squares reconstruction (Pr^T Pr)^{-1} Pr^T
 *   Sg[k][j] = int over subcell j of phi_k = Pr[j][k] / S */
typedef struct {
    int n, S;
    double Pr[(2 * ORC_MAXN - 1) * ORC_MAXN], Rc[ORC_MAXN * (2 * ORC_MAXN - 1)];
} subcell_ops;

static int make_subcell_ops(const basis *b, subcell_ops *o)
{
    const int n = b->n, S = 2 * n - 1;
    o->n = n;
    o->S = S;
    double xq[ORC_MAXN], wq[ORC_MAXN], phi[ORC_MAXN];
    if (orc_gauss_legendre(n, xq, wq)) return -1;
    for (int j = 0; j < S; ++j) {
        for (int k = 0; k < n; ++k) o->Pr[j * n + k] = 0.0;
        for (int q = 0; q < n; ++q) {
            orc_lagrange_eval(n, b->x, (j + xq[q]) / S, phi);
            for (int k = 0; k < n; ++k) o->Pr[j * n + k] += wq[q] * phi[k];
        }
    }
    /* normal equations: (Pr^T Pr) Rc = Pr^T */
    double A[ORC_MAXN * ORC_MAXN];
    int piv[ORC_MAXN];
    for (int k = 0; k < n; ++k)
        for (int l = 0; l < n; ++l) {
            double a = 0.0;
            for (int j = 0; j < S; ++j) a += o->Pr[j * n + k] * o->Pr[j * n + l];
            A[k * n + l] = a;
        }
    if (lu_factor(n, A, piv)) return -1;
    for (int j = 0; j < S; ++j) {
        double col[ORC_MAXN];
        for (int k = 0; k < n; ++k) col[k] = o->Pr[j * n + k];
        lu_solve(n, A, piv, col);
        for (int k = 0; k < n; ++k) o->Rc[k * S + j] = col[k];
    }
    return 0;
}

/* Subcell averages of one element's nodal state: avg[sub][v] =
 * sum_s prod_d Pr[sub_d][s_d] u[s][v] (S^d x m). */
static void subcell_averages(const orc_cfg *c, const subcell_ops *o, const double *u, double *avg)
{
    const int n = o->n, S = o->S, dim = c->dim, m = c->m, ns = ipow(n, dim), nsub = ipow(S, dim);
    for (int a = 0; a < nsub; ++a)
        for (int v = 0; v < m; ++v) {
            double acc = 0.0;
            for (int s = 0; s < ns; ++s) {
                double wgt = 1.0;
                for (int d = 0; d < dim; ++d) wgt *= o->Pr[digit(a, S, d) * n + digit(s, n, d)];
                acc += wgt * u[(size_t)s * m + v];
            }
            avg[(size_t)a * m + v] = acc;
        }
}

/* Nodal state from subcell averages by least squares (R28). */
static void subcell_reconstruct(const orc_cfg *c, const subcell_ops *o, const double *avg, double *u)
{
    const int n = o->n, S = o->S, dim = c->dim, m = c->m, ns = ipow(n, dim), nsub = ipow(S, dim);
    for (int s = 0; s < ns; ++s)
        for (int v = 0; v < m; ++v) {
            double acc = 0.0;
            for (int a = 0; a < nsub; ++a) {
                double wgt = 1.0;
                for (int d = 0; d < dim; ++d) wgt *= o->Rc[digit(s, n, d) * S + digit(a, S, d)];
                acc += wgt * avg[(size_t)a * m + v];
            }
            u[(size_t)s * m + v] = acc;
        }
}

/* Euler admissibility: positive density and pressure. */
static int euler_admissible(const orc_cfg *c, const double *q)
{
    if (c->pde != 2) return 1;
    const double rho = q[0];
    double kin = 0.0;
    for (int k = 0; k < c->dim; ++k) kin += q[1 + k] * q[1 + k];
    const double p = (c->prm[0] - 1.0) * (q[c->dim + 1] - 0.5 * kin / rho);
    return rho > 0.0 && p > 0.0;
}

static double minmod(double a, double b)
{
    if (a * b <= 0.0) return 0.0;
    return fabs(a) < fabs(b) ? a : b;
}

/* Exported for the pins: the 1D subcell operators of degree N
 * (Pr: (2N+1) x (N+1), Rc: (N+1) x (2N+1)). */
int orc_subcell_ops(int N, double *Pr, double *Rc)
{
    basis b;
    subcell_ops o;
    if (make_basis(N, &b) || make_subcell_ops(&b, &o)) return -1;
    memcpy(Pr, o.Pr, sizeof(double) * o.S * o.n);
    memcpy(Rc, o.Rc, sizeof(double) * o.n * o.S);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Whole-mesh operations on the periodic Cartesian grid                      */
/* ------------------------------------------------------------------------ */

static long n_elems(const orc_cfg *c)
{
    long E = 1;
    for (int d = 0; d < c->dim; ++d) E *= c->cells[d];
    return E;
}

/* neighbour of element e in direction d, offset +1 or -1, periodic wrap */
static long neighbour(const orc_cfg *c, long e, int d, int off)
{
    long idx[3] = {0, 0, 0}, r = e;
    for (int k = 0; k < c->dim; ++k) { idx[k] = r % c->cells[k]; r /= c->cells[k]; }
    idx[d] = (idx[d] + off + c->cells[d]) % c->cells[d];
    long out = 0;
    for (int k = c->dim - 1; k >= 0; --k) out = out * c->cells[k] + idx[k];
    return out;
}

/* lambda_d^max over all nodes of U, per direction d */
void orc_max_eigs(const orc_cfg *c, const double *U, double *lmax)
{
    long E = n_elems(c);
    int ns = ipow(c->N + 1, c->dim);
    for (int d = 0; d < c->dim; ++d) {
        double mx = 0.0;
        for (long i = 0; i < E * ns; ++i) {
            double l = orc_max_eig(c, &U[(size_t)i * c->m], d);
            if (l > mx) mx = l;
        }
        lmax[d] = mx;
    }
}

/* CFL condition of Sec. 3: dt = alpha / sum_d lambda_d^max / dx_d */
double orc_cfl_dt(const orc_cfg *c, const double *U)
{
    double lmax[3];
    orc_max_eigs(c, U, lmax);
    double S = 0.0;
    for (int d = 0; d < c->dim; ++d) S += lmax[d] / cell_dx(c, d);
    return orc_alpha(c) / S;
}

/* Subcell data of element e at t^n (eq. subcellaverage): the averages of
 * its nodal state U0, or (R35) the subcell averages it kept from the step
 * that limited it, sub[e] ([nsub][m]), where kept[e] is set.  sub and kept
 * may be NULL (nothing kept). */
static void un_averages(const orc_cfg *c, const subcell_ops *o, const double *U0, const double *sub,
                        const int *kept, long e, double *avg)
{
    const int ns = ipow(o->n, c->dim), nsub = ipow(o->S, c->dim), m = c->m;
    if (sub && kept && kept[e])
        memcpy(avg, &sub[(size_t)e * nsub * m], sizeof(double) * (size_t)nsub * m);
    else
        subcell_averages(c, o, &U0[(size_t)e * ns * m], avg);
}

/* Steps 1 and 2 of the limiter (R25): extreme subcell averages of the
 * state U0 at t^n per element and variable (with the kept data of R35
 * where sub / kept give them), then the troubled elements of the candidate
 * U -> bad[e].  Returns their number, or < 0 on failure. */
static long detect_troubled(const orc_cfg *c, const subcell_ops *so, const double *U0, const double *sub,
                            const int *kept, const double *U, int *bad)
{
    const subcell_ops o = *so;
    const int n = o.n, dim = c->dim, m = c->m;
    const int ns = ipow(n, dim), nsub = ipow(o.S, dim);
    const long E = n_elems(c);
    double *mm = malloc(sizeof(double) * (size_t)E * m * 2);          /* [e][v][min|max] of U0 */
    if (!mm) return -2;
    long count = 0;

    /* 1. extreme subcell averages of u^n */
#pragma omp parallel
    {
        double *avg = malloc(sizeof(double) * (size_t)nsub * m);
#pragma omp for schedule(static)
        for (long e = 0; e < E; ++e) {
            un_averages(c, &o, U0, sub, kept, e, avg);
            for (int v = 0; v < m; ++v) {
                double lo = avg[v], hi = avg[v];
                for (int a = 1; a < nsub; ++a) {
                    const double x = avg[(size_t)a * m + v];
                    lo = x < lo ? x : lo;
                    hi = x > hi ? x : hi;
                }
                mm[((size_t)e * m + v) * 2] = lo;
                mm[((size_t)e * m + v) * 2 + 1] = hi;
            }
        }
        free(avg);
    }
    /* 2. detection on the candidate */
#pragma omp parallel
    {
        double *avg = malloc(sizeof(double) * (size_t)nsub * m);
#pragma omp for schedule(static) reduction(+ : count)
        for (long e = 0; e < E; ++e) {
            const double *u = &U[(size_t)e * ns * m];
            int t = 0;
            for (size_t i = 0; i < (size_t)ns * m; ++i) t |= !isfinite(u[i]);
            for (int s = 0; s < ns && !t; ++s) t |= !euler_admissible(c, &u[(size_t)s * m]);
            if (!t) {
                subcell_averages(c, &o, u, avg);
                for (int a = 0; a < nsub && !t; ++a) t |= !euler_admissible(c, &avg[(size_t)a * m]);
                for (int v = 0; v < m && !t; ++v) {
                    double lo = mm[((size_t)e * m + v) * 2], hi = mm[((size_t)e * m + v) * 2 + 1];
                    for (int d = 0; d < dim; ++d)
                        for (int off = -1; off <= 1; off += 2) {
                            const long nb = neighbour(c, e, d, off);
                            lo = fmin(lo, mm[((size_t)nb * m + v) * 2]);
                            hi = fmax(hi, mm[((size_t)nb * m + v) * 2 + 1]);
                        }
                    const double delta = fmax(1e-4, 1e-3 * (hi - lo));
                    for (int a = 0; a < nsub && !t; ++a) {
                        const double x = avg[(size_t)a * m + v];
                        t |= x < lo - delta || x > hi + delta;
                    }
                }
            }
            bad[e] = t;
            count += t;
        }
        free(avg);
    }
    free(mm);
    return count;
}

/* The a posteriori subcell limiter (Sec. 2.3) on a candidate U (in place),
 * from the state U0 at t^n and the candidate's traces qf / ff:
 *   1. extreme subcell averages of U0 per element and variable;
 *   2. detection (R25) -> troubled[e] (may be NULL);
 *   3. troubled elements: MUSCL-Hancock on their subcells from U0 (R26,
 *      R29), least-squares reconstruction (R28), boundary subcell
 *      fluctuations kept (the one each face neighbour receives);
 *   4. unlimited face neighbours of troubled elements: their DG face flux on
 *      the common face replaced by the projected subcell fluxes (R27).
 * Returns the number of troubled elements, or < 0 on failure. */
static long apply_limiter(const orc_cfg *c, const basis *b, const double *U0, double *U, const double *qf,
                          const double *ff, double dt, int *troubled, double *sub, int *kept)
{
    subcell_ops o;
    if (make_subcell_ops(b, &o)) return -1;
    const int n = b->n, S = o.S, dim = c->dim, m = c->m;
    const int ns = ipow(n, dim), nf = ipow(n, dim - 1), nsub = ipow(S, dim), nline = ipow(S, dim - 1);
    const long E = n_elems(c);
    const size_t fsz = (size_t)2 * dim * nf * m;
    const int ncp = c->pde == 4, src = c->pde == 1, mev = orc_nevolved(c);
    int *bad = malloc(sizeof(int) * (size_t)E);
    double *Unew = malloc(sizeof(double) * (size_t)E * ns * m);
    /* [e][d][side][line][2m]: the boundary fluctuation a face neighbour
     * receives, then that neighbour's own subcell state at the face */
    double *Fb = malloc(sizeof(double) * (size_t)E * dim * 2 * nline * 2 * m);
    /* R35: the troubled elements' new subcell averages, kept for the next
     * step (written to sub once every element has read its u^n data) */
    double *Snew = sub ? malloc(sizeof(double) * (size_t)E * nsub * m) : NULL;
    if (!bad || !Unew || !Fb || (sub && !Snew)) { free(bad); free(Unew); free(Fb); free(Snew); return -2; }
    const long count = detect_troubled(c, &o, U0, sub, kept, U, bad);
    if (count < 0) { free(bad); free(Unew); free(Fb); free(Snew); return count; }

    /* 3. subcell finite-volume step of the troubled elements */
#pragma omp parallel
    {
        double *avg = malloc(sizeof(double) * (size_t)(1 + 2 * dim) * nsub * m);
        double *dq = malloc(sizeof(double) * (size_t)nsub * m);
        double *ctr = malloc(sizeof(double) * (size_t)nsub * m);  /* sum over d of the half-step changes */
#pragma omp for schedule(dynamic)
        for (long e = 0; e < E; ++e) {
            if (!bad[e]) continue;
            /* slot 0: e; 1 + 2d + (0|1): the neighbour -1 / +1 along d */
            un_averages(c, &o, U0, sub, kept, e, avg);
            for (int d = 0; d < dim; ++d)
                for (int sd = 0; sd < 2; ++sd)
                    un_averages(c, &o, U0, sub, kept, neighbour(c, e, d, sd ? 1 : -1),
                                &avg[(size_t)(1 + 2 * d + sd) * nsub * m]);
            for (size_t i = 0; i < (size_t)nsub * m; ++i) dq[i] = ctr[i] = 0.0;
            for (int d = 0; d < dim; ++d) {
                const double h = cell_dx(c, d) / S, r = dt / h;
                for (int l = 0; l < nline; ++l) {
                    /* the line of subcells along d through transverse index l */
                    int base = 0, pw = 1, rem = l;
                    for (int k = 0; k < dim; ++k) {
                        if (k != d) { base += (rem % S) * pw; rem /= S; }
                        pw *= S;
                    }
                    const int st = ipow(S, d);
                    double line[2 * ORC_MAXN + 3][ORC_MAXM];  /* cells -2 .. S+1 */
                    for (int i = -2; i <= S + 1; ++i) {
                        const double *src;
                        if (i < 0) src = &avg[((size_t)(1 + 2 * d) * nsub + base + (S + i) * st) * m];
                        else if (i >= S) src = &avg[((size_t)(2 + 2 * d) * nsub + base + (i - S) * st) * m];
                        else src = &avg[((size_t)base + i * st) * m];
                        memcpy(line[i + 2], src, sizeof(double) * m);
                    }
                    double qm[2 * ORC_MAXN + 1][ORC_MAXM], qp[2 * ORC_MAXN + 1][ORC_MAXM];  /* cells -1 .. S */
                    double cs[2 * ORC_MAXN + 1][ORC_MAXM], cw[2 * ORC_MAXN + 1][ORC_MAXM];  /* cells 0 .. S-1: */
                    double cc[2 * ORC_MAXN + 1][ORC_MAXM];  /* slope, half-step centre, its change without S */
                    for (int i = -1; i <= S; ++i) {
                        double lo[ORC_MAXM], hi[ORC_MAXM], fl[ORC_MAXM], fh[ORC_MAXM], sl[ORC_MAXM];
                        double Bs[ORC_MAXM], Sv[ORC_MAXM];
                        for (int v = 0; v < m; ++v) {
                            sl[v] = minmod(line[i + 2][v] - line[i + 1][v], line[i + 3][v] - line[i + 2][v]);
                            lo[v] = line[i + 2][v] - 0.5 * sl[v];
                            hi[v] = line[i + 2][v] + 0.5 * sl[v];
                        }
                        orc_flux(c, lo, d, fl);
                        orc_flux(c, hi, d, fh);
                        if (ncp) orc_ncp(c, line[i + 2], d, sl, Bs);          /* B_d(w) times the slope */
                        if (src) orc_source(c, line[i + 2], Sv);
                        for (int v = 0; v < m; ++v) {
                            const double df = ncp ? fh[v] - fl[v] + Bs[v] : fh[v] - fl[v];
                            qm[i + 1][v] = lo[v] - 0.5 * r * df;
                            qp[i + 1][v] = hi[v] - 0.5 * r * df;
                            if (src) {
                                qm[i + 1][v] += 0.5 * dt * Sv[v];
                                qp[i + 1][v] += 0.5 * dt * Sv[v];
                            }
                            if (i >= 0 && i < S) {
                                cs[i][v] = sl[v];
                                cc[i][v] = -0.5 * r * df;
                                cw[i][v] = line[i + 2][v] + cc[i][v] + (src ? 0.5 * dt * Sv[v] : 0.0);
                            }
                        }
                    }
                    /* faces 0 .. S (face f: cells f-1 | f); the lower cell
                     * receives Fl, the upper one Fu (equal without B) */
                    double Fl[2 * ORC_MAXN + 1][ORC_MAXM], Fu[2 * ORC_MAXN + 1][ORC_MAXM];
                    for (int f = 0; f <= S; ++f) {
                        double fl[ORC_MAXM], fr[ORC_MAXM];
                        orc_flux(c, qp[f], d, fl);
                        orc_flux(c, qm[f + 1], d, fr);
                        if (ncp) {
                            orc_face_flux(c, d, qp[f], fl, qm[f + 1], fr, Fl[f], Fu[f]);
                        } else {
                            orc_rusanov(c, d, qp[f], fl, qm[f + 1], fr, Fl[f]);
                            memcpy(Fu[f], Fl[f], sizeof(double) * m);
                        }
                    }
                    for (int i = 0; i < S; ++i) {
                        double Bc[ORC_MAXM];
                        /* the smooth part of B(q) grad q inside the subcell, at the half-step centre */
                        if (ncp) orc_ncp(c, cw[i], d, cs[i], Bc);
                        for (int v = 0; v < m; ++v) {
                            const size_t k = ((size_t)base + i * st) * m + v;
                            dq[k] -= r * (Fl[i + 1][v] - Fu[i][v]);
                            if (ncp) dq[k] -= r * Bc[v];
                            if (src) ctr[k] += cc[i][v];
                        }
                    }
                    for (int v = 0; v < m; ++v) {
                        double *b0 = &Fb[((((size_t)e * dim + d) * 2 + 0) * nline + l) * 2 * m];
                        double *b1 = &Fb[((((size_t)e * dim + d) * 2 + 1) * nline + l) * 2 * m];
                        b0[v] = Fl[0][v];
                        b0[m + v] = qp[0][v];
                        b1[v] = Fu[S][v];
                        b1[m + v] = qm[S + 1][v];
                    }
                }
            }
            if (src) {
                /* the source at the half-step centre of all directions (second order in time) */
                for (int a = 0; a < nsub; ++a) {
                    double S0[ORC_MAXM], S1[ORC_MAXM], w[ORC_MAXM];
                    orc_source(c, &avg[(size_t)a * m], S0);
                    for (int v = 0; v < m; ++v) w[v] = avg[(size_t)a * m + v] + ctr[(size_t)a * m + v] + 0.5 * dt * S0[v];
                    orc_source(c, w, S1);
                    for (int v = 0; v < m; ++v) dq[(size_t)a * m + v] += dt * S1[v];
                }
            }
            for (size_t i = 0; i < (size_t)nsub * m; ++i) dq[i] += avg[i];
            if (Snew) memcpy(&Snew[(size_t)e * nsub * m], dq, sizeof(double) * (size_t)nsub * m);
            subcell_reconstruct(c, &o, dq, &Unew[(size_t)e * ns * m]);
            /* the material fields obey q_t = 0: kept as they were */
            for (int s2 = 0; s2 < ns; ++s2)
                for (int v = mev; v < m; ++v)
                    Unew[((size_t)e * ns + s2) * m + v] = U0[((size_t)e * ns + s2) * m + v];
        }
        free(avg);
        free(dq);
        free(ctr);
    }
    /* 4. unlimited neighbours: projected subcell fluxes on the common faces */
#pragma omp parallel for schedule(static)
    for (long e = 0; e < E; ++e) {
        if (bad[e]) continue;
        for (int d = 0; d < dim; ++d)
            for (int side = 0; side < 2; ++side) {
                const long nb = neighbour(c, e, d, side ? 1 : -1);
                if (!bad[nb]) continue;
                /* the troubled neighbour's boundary fluxes on this face: its
                 * side 0 face if e is below it (side 1 of e), else side 1 */
                const double *Fs = &Fb[(((size_t)nb * dim + d) * 2 + (side ? 0 : 1)) * nline * 2 * m];
                for (int p = 0; p < nf; ++p) {
                    /* the face node's transverse indices */
                    int pk[3], rem = p, kk = 0;
                    for (int k = 0; k < dim; ++k) {
                        if (k == d) continue;
                        pk[kk++] = rem % n;
                        rem /= n;
                    }
                    /* the DG flux this element used on the face */
                    double lower[ORC_MAXM], upper[ORC_MAXM];
                    const long el = side ? e : nb, eu = side ? nb : e;
                    const size_t oL = (size_t)el * fsz + (((size_t)d * 2 + 1) * nf + p) * m;
                    const size_t oR = (size_t)eu * fsz + (((size_t)d * 2 + 0) * nf + p) * m;
                    orc_face_flux(c, d, &qf[oL], &ff[oL], &qf[oR], &ff[oR], lower, upper);
                    const double *Fdg = side ? lower : upper;
                    const double *qown = side ? &qf[oL] : &qf[oR];
                    double Ft[ORC_MAXM];
                    for (int v = 0; v < m; ++v) Ft[v] = 0.0;
                    for (int l = 0; l < nline; ++l) {
                        double wgt = 1.0;
                        int lr = l;
                        for (int k = 0; k < dim - 1; ++k) {
                            const int j = lr % S;
                            lr /= S;
                            wgt *= o.Pr[j * n + pk[k]] / S / b->w[pk[k]];
                        }
                        const double *fs = &Fs[(size_t)l * 2 * m];
                        if (ncp) {
                            /* R30: plus the path integral from this element's
                             * own DG trace to its own subcell state at the face */
                            double J[ORC_MAXM];
                            orc_path_jump(c, d, qown, fs + m, J);
                            for (int v = 0; v < m; ++v) Ft[v] += wgt * (fs[v] + J[v]);
                        } else {
                            for (int v = 0; v < m; ++v) Ft[v] += wgt * fs[v];
                        }
                    }
                    for (int s = 0; s < ns; ++s) {
                        if (face_index(s, n, dim, d) != p) continue;
                        const int sd = digit(s, n, d);
                        const double lift = (side ? b->F1[sd] : -b->F0[sd]) / (cell_dx(c, d) * b->w[sd]);
                        for (int v = 0; v < m; ++v) U[((size_t)e * ns + s) * m + v] -= dt * lift * (Ft[v] - Fdg[v]);
                    }
                }
            }
    }
    for (long e = 0; e < E; ++e) {
        if (bad[e]) memcpy(&U[(size_t)e * ns * m], &Unew[(size_t)e * ns * m], sizeof(double) * ns * m);
        if (troubled) troubled[e] = bad[e];
        if (Snew && bad[e]) memcpy(&sub[(size_t)e * nsub * m], &Snew[(size_t)e * nsub * m], sizeof(double) * nsub * m);
        if (kept) kept[e] = bad[e];
    }
    free(bad); free(Unew); free(Fb); free(Snew);
    return count;
}

/* One ADER-DG step with the given dt: predictor on every element, Rusanov
 * on every face, corrector (eq. pde.nc.gw2).  U is overwritten with u^{n+1}.
 * If V_out/qf_out/ff_out are non-NULL, the per-element volume terms and
 * traces are copied there (E n^d m and E 2d n^{d-1} m). */
/* Predictors of the previous step, for the extrapolation guess: qhat of
 * every element ([E][n][n^d][m]) and the step it covered. */
typedef struct {
    double *prev, *next;  /* read this step / written this step */
    double dt_prev;
    int valid;            /* prev holds a previous step */
} history;

static int step_impl(const orc_cfg *c, double *U, double dt, double *V_out, double *qf_out, double *ff_out,
                     history *h, int *troubled, long *ntroubled, double *sub, int *kept)
{
    basis b;
    if (make_basis(c->N, &b)) return -1;
    /* the limiter needs every step's predictor fresh (no extrapolation) */
    if (c->limiter && c->guess == 3) return -3;
    const int n = b.n, dim = c->dim, m = c->m;
    const int ns = ipow(n, dim), nf = ipow(n, dim - 1);
    const long E = n_elems(c);
    const size_t fsz = (size_t)2 * dim * nf * m;
    double *V = malloc(sizeof(double) * (size_t)E * ns * m);
    double *qf = malloc(sizeof(double) * (size_t)E * fsz);
    double *ff = malloc(sizeof(double) * (size_t)E * fsz);
    double *U0 = c->limiter ? malloc(sizeof(double) * (size_t)E * ns * m) : NULL;
    if (!V || !qf || !ff || (c->limiter && !U0)) { free(V); free(qf); free(ff); free(U0); return -2; }
    if (U0) memcpy(U0, U, sizeof(double) * (size_t)E * ns * m);
    int err = 0;

#pragma omp parallel
    {
        double *work = malloc(sizeof(double) * predictor_work_len(c));
        double *qbar = malloc(sizeof(double) * (size_t)ns * m);
        double *Fbar = malloc(sizeof(double) * (size_t)dim * ns * m);
        if (!work || !qbar || !Fbar) {
#pragma omp atomic write
            err = -2;
        } else {
#pragma omp for schedule(static)
            for (long e = 0; e < E; ++e) {
                const size_t qoff = (size_t)e * n * ns * m;
                predictor_elem(c, &b, &U[(size_t)e * ns * m], dt, h ? &h->next[qoff] : NULL, qbar, Fbar, work,
                               (h && h->valid) ? &h->prev[qoff] : NULL, (h && h->valid) ? dt / h->dt_prev : 1.0);
                volume_elem(c, &b, Fbar, &V[(size_t)e * ns * m]);
                if (has_nc_or_source(c)) volume_nc_elem(c, &b, work, &V[(size_t)e * ns * m], work + (size_t)n * ns * m);
                traces_elem(c, &b, qbar, Fbar, &qf[(size_t)e * fsz], &ff[(size_t)e * fsz]);
            }
        }
        free(work); free(qbar); free(Fbar);
    }
    if (err) { free(V); free(qf); free(ff); return err; }

#pragma omp parallel for schedule(static)
    for (long e = 0; e < E; ++e) {
        double Fm[3][ORC_MAXN * ORC_MAXN * ORC_MAXM], Fp[3][ORC_MAXN * ORC_MAXN * ORC_MAXM];
        double other[ORC_MAXM];
        for (int d = 0; d < dim; ++d) {
            long em = neighbour(c, e, d, -1), ep = neighbour(c, e, d, +1);
            for (int p = 0; p < nf; ++p) {
                /* face at xi_d = 0: lower = em (its side 1), upper = e (its side 0) */
                size_t oL = (size_t)em * fsz + (((size_t)d * 2 + 1) * nf + p) * m;
                size_t oR = (size_t)e * fsz + (((size_t)d * 2 + 0) * nf + p) * m;
                orc_face_flux(c, d, &qf[oL], &ff[oL], &qf[oR], &ff[oR], other, &Fm[d][(size_t)p * m]);
                /* face at xi_d = 1: lower = e (side 1), upper = ep (side 0) */
                oL = (size_t)e * fsz + (((size_t)d * 2 + 1) * nf + p) * m;
                oR = (size_t)ep * fsz + (((size_t)d * 2 + 0) * nf + p) * m;
                orc_face_flux(c, d, &qf[oL], &ff[oL], &qf[oR], &ff[oR], &Fp[d][(size_t)p * m], other);
            }
        }
        for (int s = 0; s < ns; ++s)
            for (int v = 0; v < m; ++v) {
                double surf = 0.0;
                for (int d = 0; d < dim; ++d) {
                    int sd = digit(s, n, d);
                    int p = face_index(s, n, dim, d);
                    surf += (b.F1[sd] * Fp[d][(size_t)p * m + v] - b.F0[sd] * Fm[d][(size_t)p * m + v])
                            / (cell_dx(c, d) * b.w[sd]);
                }
                size_t i = ((size_t)e * ns + s) * m + v;
                U[i] = U[i] + dt * (V[i] - surf);
            }
    }
    if (c->limiter) {
        const long cnt = apply_limiter(c, &b, U0, U, qf, ff, dt, troubled, sub, kept);
        if (cnt < 0) err = (int)cnt;
        if (ntroubled) *ntroubled = cnt;
    }
    if (V_out) memcpy(V_out, V, sizeof(double) * (size_t)E * ns * m);
    if (qf_out) memcpy(qf_out, qf, sizeof(double) * (size_t)E * fsz);
    if (ff_out) memcpy(ff_out, ff, sizeof(double) * (size_t)E * fsz);
    free(V); free(qf); free(ff); free(U0);
    return err;
}

int orc_step_ex(const orc_cfg *c, double *U, double dt, double *V_out, double *qf_out, double *ff_out)
{
    return step_impl(c, U, dt, V_out, qf_out, ff_out, NULL, NULL, NULL, NULL, NULL);
}

int orc_step(const orc_cfg *c, double *U, double dt) { return orc_step_ex(c, U, dt, NULL, NULL, NULL); }

/* One step with the limiter's outcome: troubled[e] (E ints) and their count. */
/* The limiter's detection alone (R25): troubled[e] of the candidate U
 * against the state U0 at t^n; returns their number, or < 0. */
long orc_detect(const orc_cfg *c, const double *U0, const double *U, int *troubled)
{
    basis b;
    subcell_ops o;
    if (make_basis(c->N, &b) || make_subcell_ops(&b, &o)) return -1;
    return detect_troubled(c, &o, U0, NULL, NULL, U, troubled);
}

int orc_step_limited(const orc_cfg *c, double *U, double dt, int *troubled, long *ntroubled)
{
    return step_impl(c, U, dt, NULL, NULL, NULL, NULL, troubled, ntroubled, NULL, NULL);
}

/* R35, kept subcell data: one limited step in which an element with
 * kept[e] set takes sub[e] ([E][(2N+1)^d][m]) as its subcell data at t^n.
 * On return the troubled elements' new subcell averages are in sub and
 * kept[e] = troubled[e] (both arrays in and out). */
int orc_step_limited_kept(const orc_cfg *c, double *U, double *sub, int *kept, double dt, int *troubled,
                          long *ntroubled)
{
    if (!c->limiter || !sub || !kept) return -1;
    return step_impl(c, U, dt, NULL, NULL, NULL, NULL, troubled, ntroubled, sub, kept);
}

/* R35: the CFL step of a state whose elements with kept[e] set are limited
 * ones: their wave speeds are those of their subcell averages sub[e], not
 * of the nodes of the reconstructed polynomial. */
double orc_cfl_dt_kept(const orc_cfg *c, const double *U, const double *sub, const int *kept)
{
    const long E = n_elems(c);
    const int ns = ipow(c->N + 1, c->dim), nsub = ipow(2 * c->N + 1, c->dim), m = c->m;
    double S = 0.0;
    for (int d = 0; d < c->dim; ++d) {
        double mx = 0.0;
        for (long e = 0; e < E; ++e) {
            const int kept_e = kept && kept[e];
            const double *q = kept_e ? &sub[(size_t)e * nsub * m] : &U[(size_t)e * ns * m];
            for (int i = 0; i < (kept_e ? nsub : ns); ++i) {
                const double l = orc_max_eig(c, &q[(size_t)i * m], d);
                if (l > mx) mx = l;
            }
        }
        S += mx / cell_dx(c, d);
    }
    return orc_alpha(c) / S;
}

/* R35: a state given by the subcell averages avg of every element
 * ([E][(2N+1)^d][m]): U = their least-squares reconstruction (R28),
 * element by element. */
int orc_subcell_init(const orc_cfg *c, const double *avg, double *U)
{
    basis b;
    subcell_ops o;
    if (make_basis(c->N, &b) || make_subcell_ops(&b, &o)) return -1;
    const long E = n_elems(c);
    const int ns = ipow(o.n, c->dim), nsub = ipow(o.S, c->dim), m = c->m;
    for (long e = 0; e < E; ++e) subcell_reconstruct(c, &o, &avg[(size_t)e * nsub * m], &U[(size_t)e * ns * m]);
    return 0;
}

/* Time loop with the CFL step and the clip to t_end:
 *   dtc = orc_cfl_dt(U);  if t + dtc >= t_end: dt = t_end - t, t = t_end
 *   else dt = dtc, t = t + dt.
 * dt_hist (nullable, length >= max_steps) receives each dt. */
static int run_impl(const orc_cfg *c, double *U, double *sub, int *kept, double t0, double t_end, long max_steps,
                    double *t_out, long *steps_out, double *dt_hist)
{
    double t = t0;
    long k = 0;
    history hist = {NULL, NULL, 0.0, 0}, *h = NULL;
    if (c->guess == 3) {  /* the extrapolation guess keeps the predictors */
        const size_t len = (size_t)n_elems(c) * ipow(c->N + 1, c->dim + 1) * c->m;
        hist.prev = malloc(sizeof(double) * len);
        hist.next = malloc(sizeof(double) * len);
        if (!hist.prev || !hist.next) { free(hist.prev); free(hist.next); return -2; }
        h = &hist;
    }
    while (t < t_end && k < max_steps) {
        double dtc = sub ? orc_cfl_dt_kept(c, U, sub, kept) : orc_cfl_dt(c, U);
        double dt, tn;
        if (t + dtc >= t_end) { dt = t_end - t; tn = t_end; }
        else { dt = dtc; tn = t + dtc; }
        int rc = step_impl(c, U, dt, NULL, NULL, NULL, h, NULL, NULL, sub, kept);
        if (rc) { if (h) { free(hist.prev); free(hist.next); } return rc; }
        if (h) {
            double *tmp = hist.prev; hist.prev = hist.next; hist.next = tmp;
            hist.dt_prev = dt;
            hist.valid = 1;
        }
        if (dt_hist) dt_hist[k] = dt;
        t = tn;
        ++k;
    }
    if (h) { free(hist.prev); free(hist.next); }
    if (t_out) *t_out = t;
    if (steps_out) *steps_out = k;
    return 0;
}

int orc_run(const orc_cfg *c, double *U, double t0, double t_end, long max_steps,
            double *t_out, long *steps_out, double *dt_hist)
{
    if (c->limiter != 2) return run_impl(c, U, NULL, NULL, t0, t_end, max_steps, t_out, steps_out, dt_hist);
    /* R35 from a nodal state: nothing kept at t0 */
    const long E = n_elems(c);
    double *sub = malloc(sizeof(double) * (size_t)E * ipow(2 * c->N + 1, c->dim) * c->m);
    int *kept = calloc((size_t)E, sizeof(int));
    if (!sub || !kept) { free(sub); free(kept); return -2; }
    const int rc = run_impl(c, U, sub, kept, t0, t_end, max_steps, t_out, steps_out, dt_hist);
    free(sub); free(kept);
    return rc;
}

/* orc_run with the kept subcell data of R35 carried in and out (sub, kept
 * as for orc_step_limited_kept). */
int orc_run_kept(const orc_cfg *c, double *U, double *sub, int *kept, double t0, double t_end, long max_steps,
                 double *t_out, long *steps_out, double *dt_hist)
{
    if (c->limiter != 2 || !sub || !kept) return -1;
    return run_impl(c, U, sub, kept, t0, t_end, max_steps, t_out, steps_out, dt_hist);
}

/* Sampled step: u^{n+1} of the listed elements only (each needs the
 * predictor of itself and its 2d neighbours).  Out: n_s x n^d x m. */
int orc_step_sampled(const orc_cfg *c, const double *U, double dt, long n_s,
                     const long *elems, double *out)
{
    basis b;
    if (make_basis(c->N, &b)) return -1;
    const int n = b.n, dim = c->dim, m = c->m;
    const int ns = ipow(n, dim), nf = ipow(n, dim - 1);
    const size_t fsz = (size_t)2 * dim * nf * m;
    int err = 0;
#pragma omp parallel
    {
        double *work = malloc(sizeof(double) * predictor_work_len(c));
        double *qbar = malloc(sizeof(double) * (size_t)ns * m);
        double *Fbar = malloc(sizeof(double) * (size_t)dim * ns * m);
        double *V = malloc(sizeof(double) * (size_t)ns * m);
        double *qf = malloc(sizeof(double) * fsz * 7);
        double *ff = malloc(sizeof(double) * fsz * 7);
        if (!work || !qbar || !Fbar || !V || !qf || !ff) {
#pragma omp atomic write
            err = -2;
        } else {
#pragma omp for schedule(static)
            for (long i = 0; i < n_s; ++i) {
                long e = elems[i];
                /* slot 0: e itself; slot 1 + 2d + (0|1): neighbour -1 / +1 along d */
                long ids[7];
                ids[0] = e;
                for (int d = 0; d < dim; ++d) { ids[1 + 2 * d] = neighbour(c, e, d, -1); ids[2 + 2 * d] = neighbour(c, e, d, +1); }
                for (int k = 0; k < 1 + 2 * dim; ++k) {
                    predictor_elem(c, &b, &U[(size_t)ids[k] * ns * m], dt, NULL, qbar, Fbar, work, NULL, 1.0);
                    if (k == 0) {
                        volume_elem(c, &b, Fbar, V);
                        if (has_nc_or_source(c)) volume_nc_elem(c, &b, work, V, work + (size_t)n * ns * m);
                    }
                    traces_elem(c, &b, qbar, Fbar, &qf[k * fsz], &ff[k * fsz]);
                }
                for (int s = 0; s < ns; ++s)
                    for (int v = 0; v < m; ++v) {
                        double surf = 0.0;
                        for (int d = 0; d < dim; ++d) {
                            int sd = digit(s, n, d), p = face_index(s, n, dim, d);
                            double fm[ORC_MAXM], fp[ORC_MAXM], other[ORC_MAXM];
                            size_t oL = 1 * fsz * (1 + 2 * d) + (((size_t)d * 2 + 1) * nf + p) * m;
                            size_t oR = (((size_t)d * 2 + 0) * nf + p) * m;
                            orc_face_flux(c, d, &qf[oL], &ff[oL], &qf[oR], &ff[oR], other, fm);
                            oL = (((size_t)d * 2 + 1) * nf + p) * m;
                            oR = fsz * (2 + 2 * d) + (((size_t)d * 2 + 0) * nf + p) * m;
                            orc_face_flux(c, d, &qf[oL], &ff[oL], &qf[oR], &ff[oR], fp, other);
                            surf += (b.F1[sd] * fp[v] - b.F0[sd] * fm[v]) / (cell_dx(c, d) * b.w[sd]);
                        }
                        size_t iu = ((size_t)e * ns + s) * m + v;
                        out[((size_t)i * ns + s) * m + v] = U[iu] + dt * (V[(size_t)s * m + v] - surf);
                    }
            }
        }
        free(work); free(qbar); free(Fbar); free(V); free(qf); free(ff);
    }
    return err;
}

/* Conserved totals M_v = sum_e |Omega_e| sum_s w_s U[e][s][v], in the fixed
 * order (e, s). */
int orc_mass(const orc_cfg *c, const double *U, double *M)
{
    basis b;
    if (make_basis(c->N, &b)) return -1;
    const int n = b.n, dim = c->dim, m = c->m, ns = ipow(n, dim);
    double vol = 1.0;
    for (int d = 0; d < dim; ++d) vol *= cell_dx(c, d);
    long E = n_elems(c);
    for (int v = 0; v < m; ++v) M[v] = 0.0;
    for (long e = 0; e < E; ++e)
        for (int s = 0; s < ns; ++s) {
            double ws = 1.0;
            for (int d = 0; d < dim; ++d) ws *= b.w[digit(s, n, d)];
            for (int v = 0; v < m; ++v) M[v] += vol * ws * U[((size_t)e * ns + s) * m + v];
        }
    return 0;
}

/* Physical coordinates of every node: X[e][s][d] (E n^d dim). */
int orc_node_coords(const orc_cfg *c, double *X)
{
    double x[ORC_MAXN], w[ORC_MAXN];
    int n = c->N + 1;
    if (orc_gauss_legendre(n, x, w)) return -1;
    const int dim = c->dim, ns = ipow(n, dim);
    long E = n_elems(c);
    for (long e = 0; e < E; ++e) {
        long r = e;
        long idx[3] = {0, 0, 0};
        for (int k = 0; k < dim; ++k) { idx[k] = r % c->cells[k]; r /= c->cells[k]; }
        for (int s = 0; s < ns; ++s)
            for (int d = 0; d < dim; ++d) {
                double h = cell_dx(c, d);
                X[((size_t)e * ns + s) * dim + d] = c->lo[d] + (idx[d] + x[digit(s, n, d)]) * h;
            }
    }
    return 0;
}

/* Sets the OpenMP thread count of later parallel loops (no-op without
 * OpenMP); n <= 0 restores the default. */
void orc_set_threads(int n)
{
#ifdef _OPENMP
    static int dflt = 0;
    if (dflt == 0) dflt = omp_get_max_threads();
    omp_set_num_threads(n > 0 ? n : dflt);
#else
    (void)n;
#endif
}

/* Number of OpenMP threads the parallel loops use (1 without OpenMP). */
int orc_threads(void)
{
#ifdef _OPENMP
    int t = 1;
#pragma omp parallel
    {
#pragma omp single
        t = omp_get_num_threads();
    }
    return t;
#else
    return 1;
#endif
}
