// Host-side construction of the 1D nodal basis of the scheme (Sec. 2.1):
// Gauss-Legendre nodes and weights on [0,1] and the small operators the
// kernels use.  Methods (chosen for robustness in double precision):
//   - nodes: eigenvalues of the symmetric tridiagonal Jacobi matrix of the
//     Legendre polynomials (Golub-Welsch), found by Sturm-sequence bisection
//   - weights: w = 2 / ((1 - y^2) P_n'(y)^2) on [-1,1], halved for [0,1]
//   - Lagrange derivative matrix and boundary values: barycentric formulas
//   - K1 = F1 F1^T - (W Dhat)^T inverted by Gauss-Jordan elimination with
//     partial pivoting.
#include <cmath>
#include <cstring>

#include "../../include/aderdg.h"
#include "basis.h"

namespace aderdg {

namespace {

// Number of eigenvalues of the n x n Jacobi matrix (zero diagonal,
// off-diagonal b_k = k / sqrt(4k^2 - 1)) that are smaller than x.
int sturm_count(int n, double x)
{
    int count = 0;
    double q = -x;  // d_1 - x with d = 0
    if (q < 0) ++count;
    for (int k = 1; k < n; ++k) {
        const double b2 = double(k) * k / (4.0 * k * k - 1.0);
        if (q == 0.0) q = 1e-300;
        q = -x - b2 / q;
        if (q < 0) ++count;
    }
    return count;
}

void legendre_and_derivative(int n, double y, double &p, double &dp)
{
    double pm1 = 1.0, pc = y;
    if (n == 0) { p = 1.0; dp = 0.0; return; }
    for (int k = 2; k <= n; ++k) {
        const double pn = ((2.0 * k - 1.0) * y * pc - (k - 1.0) * pm1) / k;
        pm1 = pc;
        pc = pn;
    }
    p = pc;
    dp = n * (pm1 - y * pc) / (1.0 - y * y);
}

}  // namespace

int gauss_legendre01(int n, double *x, double *w)
{
    if (n < 1 || n > 16) return -1;
    for (int k = 0; k < n; ++k) {
        // k-th smallest eigenvalue in (-1, 1): bisection on the Sturm count
        double lo = -1.0, hi = 1.0;
        for (int it = 0; it < 200 && hi - lo > 0.0; ++it) {
            const double mid = 0.5 * (lo + hi);
            if (mid == lo || mid == hi) break;
            if (sturm_count(n, mid) > k) hi = mid; else lo = mid;
        }
        const double y = 0.5 * (lo + hi);
        double p, dp;
        legendre_and_derivative(n, y, p, dp);
        x[k] = 0.5 * (1.0 + y);
        w[k] = 1.0 / ((1.0 - y * y) * dp * dp);
    }
    return 0;
}

int build_basis(int N, Basis &b)
{
    const int n = N + 1;
    if (n < 1 || n > NMAX) return -1;
    std::memset(&b, 0, sizeof(b));
    b.n = n;
    double x[NMAX], bw[NMAX];
    if (gauss_legendre01(n, x, b.w)) return -1;
    for (int k = 0; k < n; ++k) b.x[k] = x[k];
    // barycentric weights bw_k = 1 / prod_{j != k} (x_k - x_j)
    for (int k = 0; k < n; ++k) {
        double prod = 1.0;
        for (int j = 0; j < n; ++j)
            if (j != k) prod *= (x[k] - x[j]);
        bw[k] = 1.0 / prod;
    }
    // Dhat[j][k] = (bw_k / bw_j) / (x_j - x_k), diagonal = - row sum
    for (int j = 0; j < n; ++j) {
        double diag = 0.0;
        for (int k = 0; k < n; ++k) {
            if (k == j) continue;
            const double v = (bw[k] / bw[j]) / (x[j] - x[k]);
            b.D[j * n + k] = v;
            diag -= v;
        }
        b.D[j * n + j] = diag;
    }
    // boundary values by the barycentric formula of the second kind
    for (int side = 0; side < 2; ++side) {
        const double xi = side ? 1.0 : 0.0;
        double den = 0.0, t[NMAX];
        for (int k = 0; k < n; ++k) { t[k] = bw[k] / (xi - x[k]); den += t[k]; }
        double *phi = side ? b.F1 : b.F0;
        for (int k = 0; k < n; ++k) phi[k] = t[k] / den;
    }
    for (int k = 0; k < n; ++k) b.inv_w[k] = 1.0 / b.w[k];
    // Kw[k][j] = w_j Dhat[j][k] / w_k
    for (int k = 0; k < n; ++k)
        for (int j = 0; j < n; ++j) b.Kw[k * n + j] = b.w[j] * b.D[j * n + k] / b.w[k];
    // K1[k][l] = F1_k F1_l - w_l Dhat[l][k]; invert by Gauss-Jordan
    double A[NMAX][2 * NMAX];
    for (int k = 0; k < n; ++k) {
        for (int l = 0; l < n; ++l) {
            A[k][l] = b.F1[k] * b.F1[l] - b.w[l] * b.D[l * n + k];
            A[k][n + l] = (k == l) ? 1.0 : 0.0;
        }
    }
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (std::fabs(A[r][c]) > std::fabs(A[piv][c])) piv = r;
        if (A[piv][c] == 0.0) return -2;
        if (piv != c)
            for (int j = 0; j < 2 * n; ++j) { double t = A[c][j]; A[c][j] = A[piv][j]; A[piv][j] = t; }
        const double ip = 1.0 / A[c][c];
        for (int j = 0; j < 2 * n; ++j) A[c][j] *= ip;
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            const double f = A[r][c];
            if (f == 0.0) continue;
            for (int j = 0; j < 2 * n; ++j) A[r][j] -= f * A[c][j];
        }
    }
    // iK1W = K1^{-1} diag(w)
    for (int t = 0; t < n; ++t)
        for (int tp = 0; tp < n; ++tp) b.iK1W[t * n + tp] = A[t][n + tp] * b.w[tp];
    return 0;
}

namespace {
// Continuous explicit Runge-Kutta schemes of the CERK guess (Sec. 2.2 names
// those of Owren and Zennaro without coefficients): stages k_i = L(u + dt
// sum_{j<i} a_ij k_j), dense output u + dt sum_i b_i(th) k_i with b_i(th) =
// sum_k beta_ik th^(k+1), of uniform order p (every rooted-tree condition
// sum_i b_i(th) Phi_i(t) = th^|t| / gamma(t), |t| <= p, holds for all th).
// Order 3: the classical fourth-order method and its cubic dense output.
// Order 4: a six-stage scheme with quartic weights (five stages cannot reach
// uniform order 4), from a numerical search over the stage matrix that kept
// max |b_i(th)| small (0.35), refined to 40 digits by Newton's method on the
// order conditions; shown here to 20 digits.
// Order 5: an eleven-stage scheme with quintic weights from the same kind of
// search (the 17 tree conditions of order <= 5; max |b_i(th)| 0.31, max
// |a_ij| 0.48), refined and shown the same way.
struct CerkScheme {
    int s, p;
    double a[CERK_SMAX][CERK_SMAX];
    double beta[CERK_SMAX][5];
};
const CerkScheme kCerkOrder3 = {
    4, 3,
    {{0}, {0.5}, {0.0, 0.5}, {0.0, 0.0, 1.0}},
    {{1.0, -1.5, 2.0 / 3.0}, {0.0, 1.0, -2.0 / 3.0}, {0.0, 1.0, -2.0 / 3.0}, {0.0, -0.5, 2.0 / 3.0}},
};
const CerkScheme kCerkOrder4 = {
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

const CerkScheme kCerkOrder5 = {
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

// the scheme of the CERK guess for degree N (cerk_stages / cerk_order)
const CerkScheme &cerk_scheme_for(int N)
{
    return cerk_stages(N) == 11 ? kCerkOrder5 : (cerk_stages(N) == 6 ? kCerkOrder4 : kCerkOrder3);
}

template <typename T>
void fill_typed(const Basis &b, Ops<T> &o)
{
    std::memset(&o, 0, sizeof(o));
    const int n = b.n;
    for (int d = 0; d < 3; ++d)
        for (int i = 0; i < n * n; ++i) {
            o.Dm[d][i] = T(-b.D[i]);
            o.Kv[d][i] = T(b.Kw[i]);
        }
    for (int i = 0; i < n * n; ++i) o.iK1W[i] = T(b.iK1W[i]);
    for (int t = 0; t < n; ++t) {
        double c = 0.0;
        for (int tp = 0; tp < n; ++tp) c += b.iK1W[t * n + tp];
        o.c1[t] = T(c);
        o.w[t] = T(b.w[t]);
        o.F0[t] = T(b.F0[t]);
        o.F1[t] = T(b.F1[t]);
        o.inv_w[t] = T(b.inv_w[t]);
        o.xi[t] = T(b.x[t]);
        o.hxi2[t] = T(0.5 * b.x[t] * b.x[t]);
        {  // CERK dense-output weights at xi_t
            const CerkScheme &cs = cerk_scheme_for(n - 1);
            for (int i = 0; i < cs.s; ++i) {
                double v = 0.0, thk = b.x[t];
                for (int k = 0; k < cs.p; ++k) {
                    v += cs.beta[i][k] * thk;
                    thk *= b.x[t];
                }
                o.ck_b[i][t] = T(v);
            }
        }
        double prod = 1.0;
        for (int j = 0; j < n; ++j)
            if (j != t) prod *= b.x[t] - b.x[j];
        o.bw[t] = T(1.0 / prod);
    }
    {
        const CerkScheme &cs = cerk_scheme_for(n - 1);
        for (int i = 0; i < cs.s; ++i)
            for (int j = 0; j < i; ++j) o.ck_a[i * (i - 1) / 2 + j] = T(cs.a[i][j]);
    }
}
}  // namespace

// Subcell operators of the limiter for n = N+1 nodes and S = 2N+1 equal
// subcells of [0, 1]: pr[j][k] = average over subcell j of the k-th nodal
// basis polynomial (n-point Gauss rule on the subcell, exact for degree N),
// rc = (pr^T pr)^{-1} pr^T (least squares), by Gauss-Jordan elimination.
void fill_subcell_ops(const Basis &b, double *pr, double *rc)
{
    const int n = b.n, S = 2 * n - 1;
    double xq[NMAX], wq[NMAX], bwt[NMAX];
    gauss_legendre01(n, xq, wq);
    for (int k = 0; k < n; ++k) {
        double prod = 1.0;
        for (int j = 0; j < n; ++j)
            if (j != k) prod *= b.x[k] - b.x[j];
        bwt[k] = 1.0 / prod;
    }
    for (int j = 0; j < S; ++j)
        for (int k = 0; k < n; ++k) {
            double acc = 0.0;
            for (int q = 0; q < n; ++q) {
                const double x = (j + xq[q]) / S;
                double phi = bwt[k];  // Lagrange polynomial k at x (product form)
                for (int i = 0; i < n; ++i)
                    if (i != k) phi *= x - b.x[i];
                acc += wq[q] * phi;
            }
            pr[j * n + k] = acc;
        }
    double A[NMAX][NMAX + 2 * NMAX - 1];
    for (int k = 0; k < n; ++k) {
        for (int l = 0; l < n; ++l) {
            double a = 0.0;
            for (int j = 0; j < S; ++j) a += pr[j * n + k] * pr[j * n + l];
            A[k][l] = a;
        }
        for (int j = 0; j < S; ++j) A[k][n + j] = pr[j * n + k];
    }
    for (int c = 0; c < n; ++c) {  // the normal matrix is symmetric positive definite: no pivoting
        const double inv = 1.0 / A[c][c];
        for (int j = 0; j < n + S; ++j) A[c][j] *= inv;
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            const double f = A[r][c];
            for (int j = 0; j < n + S; ++j) A[r][j] -= f * A[c][j];
        }
    }
    for (int k = 0; k < n; ++k)
        for (int j = 0; j < S; ++j) rc[k * S + j] = A[k][n + j];
}

void fill_ops(KParams &kp)
{
    fill_typed<double>(kp.b, kp.od);
    fill_typed<float>(kp.b, kp.of);
    fill_subcell_ops(kp.b, kp.lim_pr, kp.lim_rc);
}

// 0.9 x the von Neumann stability limit of the scheme for 1D linear
// advection (limits 0.3335, 0.1709, 0.1040, 0.0699, 0.0501, 0.0377, 0.0294,
// 0.0236, 0.0193 for N = 1..9); the paper bounds alpha by 1/(2N+1) only.
double default_alpha(int N)
{
    static const double a[10] = {0.9, 0.3001, 0.1538, 0.0936, 0.0629,
                                 0.0451, 0.0339, 0.0265, 0.0212, 0.0174};
    if (N >= 0 && N <= 9) return a[N];
    return 0.5 / (2.0 * N + 1.0);
}

int pde_nvar(int kind, int dim)
{
    if (kind == 1) return 1;
    if (kind == 2) return dim + 2;
    if (kind == 3) return 9;  // compiled for d = 3 only
    if (kind == 4) return dim == 3 ? 13 : (dim == 2 ? 9 : -1);
    return -1;
}

void fill_pde_consts(int kind, PdeParams &P)
{
    for (int i = 0; i < 8; ++i) P.c[i] = 0.0;
    if (kind == 1) {  // advection
        for (int d = 0; d < 3; ++d) {
            P.c[d] = P.p[d];
            P.c[3 + d] = std::fabs(P.p[d]);
        }
        P.c[6] = -P.p[3];  // source coefficient -kappa
    } else if (kind == 2) {  // Euler
        P.c[0] = P.p[0] - 1.0;
        P.c[1] = P.p[0];
    } else if (kind == 3) {  // elasticity
        P.c[0] = 1.0 / P.p[0];
        P.c[1] = P.p[1];
        P.c[2] = P.p[2];
        P.c[3] = P.p[1] + 2.0 * P.p[2];
        P.c[4] = std::sqrt((P.p[1] + 2.0 * P.p[2]) / P.p[0]);
    }
    for (int i = 0; i < 8; ++i) P.cf[i] = (float)P.c[i];
}

int check_mesh(const aderdg_mesh_t &mesh, int kind, long long *E, const char **why)
{
    auto bad = [&](const char *m) { *why = m; return ADERDG_E_INVAL; };
    if (mesh.dim < 2 || mesh.dim > 3) return bad("dim must be 2 or 3");
    if (pde_nvar(kind, mesh.dim) < 0) return bad("unknown pde kind for this dimension");
    long long e = 1;
    for (int d = 0; d < mesh.dim; ++d) {
        // each factor <= 2^30 and the running product <= 2^31: no overflow
        if (mesh.cells[d] <= 0 || mesh.cells[d] > (1LL << 30)) return bad("bad cell count (1 .. 2^30 per direction)");
        if (!(mesh.hi[d] > mesh.lo[d]) || !std::isfinite(mesh.hi[d] - mesh.lo[d])) return bad("hi must exceed lo");
        e *= mesh.cells[d];
        if (e > (1LL << 31)) return bad("too many elements (at most 2^31)");
    }
    *E = e;
    return ADERDG_OK;
}

int check_pde_params(const aderdg_pde_t &pde, const char **why)
{
    auto bad = [&](const char *m) { *why = m; return ADERDG_E_INVAL; };
    const double *p = pde.p;
    if (pde.kind == 1 && !(std::isfinite(p[0]) && std::isfinite(p[1]) && std::isfinite(p[2]) && p[3] >= 0.0 &&
                           std::isfinite(p[3])))
        return bad("advection: finite velocity and kappa >= 0 required");
    if (pde.kind == 2 && !(p[0] > 1.0 && std::isfinite(p[0]))) return bad("gamma must be > 1");
    if (pde.kind == 3 && !(p[0] > 0 && p[2] > 0 && p[1] + 2 * p[2] > 0 && std::isfinite(p[0]) &&
                           std::isfinite(p[1]) && std::isfinite(p[2])))
        return bad("bad elastic parameters (rho > 0, mu > 0, lambda + 2 mu > 0)");
    return ADERDG_OK;
}

int check_problem(const aderdg_mesh_t &mesh, const aderdg_pde_t &pde, long long *E, const char **why)
{
    const int rc = check_mesh(mesh, pde.kind, E, why);
    return rc ? rc : check_pde_params(pde, why);
}

void fill_desc_lift(SolveDesc &sd, int N)
{
    Basis b;
    std::memset(&b, 0, sizeof(b));
    if (build_basis(N, b)) return;
    for (int d = 0; d < 3; ++d)
        for (int k = 0; k < NMAX; ++k) {
            sd.lift_f[0][d][k] = k < b.n ? (float)(sd.inv_dx[d] * b.inv_w[k] * b.F0[k]) : 0.f;
            sd.lift_f[1][d][k] = k < b.n ? (float)(sd.inv_dx[d] * b.inv_w[k] * b.F1[k]) : 0.f;
        }
}

int default_picard(int N, int guess)
{
    if (guess == 3) return 2;  // a degree-N guess: one iteration, plus one
    const int k = guess == 1 ? 1 : (guess == 2 ? 2 : (guess == 4 ? cerk_order(N) : 0));
    return N + 1 - k < 1 ? 1 : N + 1 - k;
}

}  // namespace aderdg
