// Shared device-side definitions of the ADER-DG library: the 1D basis
// passed to every kernel, the per-solve device control block, the PDE
// functions and the kernel parameter block.
//
// Notation (Dumbser et al. 2018, Sec. 2.1-2.2): n = N+1 Gauss-Legendre
// nodes xi_k and weights w_k on [0,1]; Lagrange basis phi_k;
//   Dhat[j][k] = phi_k'(xi_j)          nodal derivative (eq. D_kl times h)
//   Kw[k][j]   = w_j Dhat[j][k] / w_k   volume-integral operator divided by
//                                       the diagonal mass (eq. pde.nc.gw2)
//   iK1W       = K1^{-1} diag(w),  K1 = F1 F1^T - (W Dhat)^T   (eq. pde.st2)
//   F0[k] = phi_k(0), F1[k] = phi_k(1).
#pragma once

#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

namespace aderdg {

constexpr int NMAX = 8;  // largest n = N+1 compiled

struct Basis {
    int n;
    double x[NMAX];            // Gauss-Legendre nodes on [0, 1]
    double w[NMAX], F0[NMAX], F1[NMAX], inv_w[NMAX];
    double D[NMAX * NMAX];     // Dhat, row-major [j][k]
    double Kw[NMAX * NMAX];    // [k][j]
    double iK1W[NMAX * NMAX];  // [t][t']
};

// Per-solve control block in device memory.  The corrector accumulates the
// wave-speed maxima of the new state into lam_acc (bit patterns of
// non-negative doubles, so integer max == double max); the dt kernel turns
// them into the next CFL step.
enum : unsigned { FLAG_NONFINITE = 1u, FLAG_DONE = 2u, FLAG_TIMEOUT = 4u };

struct Control {
    double t;          // time of the state after the step in flight
    double t_end;
    double dt;         // dt of the step in flight (0: no step)
    double dt_prev;    // dt of the step before it (0: none; extrapolation guess)
    double alpha;
    double inv_dx[3];
    int dim;
    int pad0;
    unsigned long long lam_acc[3];  // max |lambda_d| of the current state
    double lam_used[3];             // maxima the last dt was computed from
    long long step;
    unsigned int flags;
    unsigned int lim_fresh;  // subcell limiter: lim_mmc holds the candidate extremes of the state's last step
    unsigned int lim_count;  // subcell limiter: troubled elements listed in lim_list this step
                             // (zeroed by the next step's dt_update)
    unsigned int lim_kept_ok;  // kept subcell data: lim_subn holds the subcell averages of the
                               // elements lim_flags marks (the last limited step, or an upload of
                               // subcell data) -- cleared by any other change of the state
};


// PDE parameters as given (aderdg_pde_t) and constants derived from them
// on the host (fill_pde_consts), in double and rounded to float, so that
// the kernels do no per-call parameter arithmetic or double->float
// conversion:
//   advection   c[d] = a_d, c[3 + d] = |a_d|
//   Euler       c[0] = gamma - 1, c[1] = gamma
//   elasticity  c[0] = 1/rho, c[1] = lambda, c[2] = mu, c[3] = lambda + 2 mu,
//               c[4] = c_p = sqrt((lambda + 2 mu) / rho)
struct PdeParams {
    double p[8];
    double c[8];
    float cf[8];
};

template <typename T>
__host__ __device__ __forceinline__ T pconst(const PdeParams &P, int i);
template <>
__host__ __device__ __forceinline__ double pconst<double>(const PdeParams &P, int i) { return P.c[i]; }
template <>
__host__ __device__ __forceinline__ float pconst<float>(const PdeParams &P, int i) { return P.cf[i]; }

// The continuous Runge-Kutta scheme of the CERK guess (Sec. 2.2) for
// degree N: the classical fourth-order method with its cubic dense output
// up to N = 4, a six-stage scheme with quartic weights at N = 5, an
// eleven-stage scheme with quintic weights from N = 6 (the degree N - 1
// that one Picard iteration wants at N = 5 and N = 6).
constexpr int CERK_SMAX = 11;
__host__ __device__ constexpr int cerk_stages(int N) { return N >= 6 ? 11 : (N >= 5 ? 6 : 4); }
__host__ __device__ constexpr int cerk_order(int N) { return N >= 6 ? 5 : (N >= 5 ? 4 : 3); }

// Operators in the compute type (filled on the host by fill_ops).  Indexed
// with compile-time constants inside unrolled loops, they are read straight
// from the kernel-parameter constant bank.  They do not depend on the mesh
// spacing, so one table serves every solve of a launch.
template <typename T>
struct Ops {
    T Dm[3][NMAX * NMAX];  // -Dhat                   [i][j] (same for every d)
    T Kv[3][NMAX * NMAX];  // Kw                      [k][j] (same for every d)
    T iK1W[NMAX * NMAX];   // K1^{-1} W               [t][t']
    T c1[NMAX];            // row sums of iK1W (time integral of a constant)
    T w[NMAX], F0[NMAX], F1[NMAX], inv_w[NMAX];
    T xi[NMAX];            // time nodes on [0, 1] (initial guesses)
    T hxi2[NMAX];          // xi^2 / 2
    T bw[NMAX];            // barycentric weights 1 / prod_{j != k} (xi_k - xi_j)
    T ck_b[CERK_SMAX][NMAX];        // CERK dense-output weights b_i(xi_t)
    T ck_a[CERK_SMAX * (CERK_SMAX - 1) / 2];  // CERK stage matrix, strictly lower triangle by rows:
                                              // a_ij at i (i - 1) / 2 + j
};

// Unsigned division by a divisor fixed for a solve (its cell counts) as a
// multiply-high and two shifts, Granlund and Montgomery, "Division by
// invariant integers using multiplication" (PLDI 1994, fig. 4.1): with
// l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1, t = mulhi(m, n),
// n / d = (t + ((n - t) >> min(l, 1))) >> max(l - 1, 0) for every 32-bit n.
struct FastDiv {
    unsigned m;
    unsigned s1, s2;
};
inline FastDiv make_fastdiv(unsigned d)
{
    unsigned l = 0;
    while (l < 32 && (1ull << l) < d) ++l;
    FastDiv f;
    f.m = (unsigned)((((1ull << l) - d) << 32) / d + 1);
    f.s1 = l < 1 ? l : 1;
    f.s2 = l > 1 ? l - 1 : 0;
    return f;
}
#ifdef __CUDACC__
__device__ __forceinline__ unsigned fdiv(unsigned n, const FastDiv &f)
{
    const unsigned t = __umulhi(n, f.m);
    return (t + ((n - t) >> f.s1)) >> f.s2;
}
#endif

// One solve of a launch (device memory).  Tiles of EPB consecutive
// elements are numbered solve after solve: this solve owns tiles
// [tile0_p, tile0_p + ceil(E / EPB_predictor)) of the predictor launch and
// likewise tile0_c for the corrector.
struct SolveDesc {
    long long E;
    long long tile0_p, tile0_c;
    int cells[3];
    int picard;        // Picard iterations after the initial guess
    int picard_first;  // extrapolation guess: iterations of a step without a previous predictor
    int guess;         // initial guess: 0 trivial, 1 second order, 2 third order,
                       // 3 extrapolation of the previous predictor, 4 CERK (Sec. 2.2)
    double inv_dx[3];
    float inv_dx_f[3]; // 1/dx_d and dx_0/dx_d in FP32 (precomputed on the host)
    float ratio_f[3];
    const double *u;   // state u^n            [E][NS][M]
    double *u_out;     // state u^{n+1} (may alias u)
    void *V;           // volume term          [E][NS][M] of T
    void *tr;          // trace records        [E][DIM][2][NF][RS] of T
    double *ref;       // FP32 path: reference state per element [E][M]; unused in FP64
    void *qprev;       // extrapolation guess: last predictor [E][n][NS][M] of T
    Control *ctl;
    // subcell limiter (either precision; the state is FP64): u^n saved
    // before the corrector, the extreme subcell averages of u^n and of the
    // candidate [E][M][2], and the troubled flags [E]
    const double *u_prev;
    double *lim_mm;
    double *lim_mmc;
    int *lim_flags;
    int *lim_list;  // the troubled elements of the step, in detection order [ctl->lim_count]
    // kept subcell data (Sec. 2.3, eq. subcellaverage, for a limited element
    // the averages its subcell scheme produced; NULL unless the handle keeps
    // them), each [E][(2N+1)^d][M]: lim_sub the subcell data of u^n of the
    // elements with lim_kept[e] set, lim_subn the new averages of this step's
    // troubled elements (k_lim_minmax moves them to lim_sub and sets lim_kept
    // at the start of the next step)
    double *lim_sub;
    double *lim_subn;
    int *lim_kept;
    // the subcell fluxes the subcell scheme forms on the element faces of the
    // first lim_fb_slots troubled elements of the step, for the coupling of
    // their unlimited neighbours ([slot][d][side][line][FB], slot = the index
    // in lim_list, FB = M values, or 2M for a non-conservative system: the
    // fluctuation the neighbour receives and the neighbour's own subcell state
    // at the face); lim_slot[e]: the slot of troubled element e.  NULL / 0:
    // the coupling forms them itself
    double *lim_fb;
    int *lim_slot;
    long long lim_fb_slots;
    // domain decomposition (a block of a partitioned mesh, see partition.cu):
    // elist: the predictor's elements, E indices into the block (its
    // boundary or its interior elements); NULL: elements 0 .. E-1.
    // halo_tr[d][side]: for the corrector, the face chunks [j][NF][RS] of the
    // neighbouring block across this block's face (d, side), j the element's
    // index over the other directions (lowest fastest), and halo_ref[d][side]
    // their FP32-path reference states [j][M]; NULL: the direction is not
    // split and wraps periodically inside the block.
    const int *elist;
    const void *halo_tr[3][2];
    const double *halo_ref[3][2];
    // FP32 path: the corrector's lift coefficients (1/dx_d) F_{0|1}[k] / w_k
    // rounded to float, [side][d][k] (fill_desc_lift)
    float lift_f[2][3][NMAX];
    // element index -> cell: divisions by cells[0] and cells[1]
    FastDiv div_cx, div_cy;
};

// the per-solve constants derived from cells and inv_dx
inline void fill_desc_spacing(SolveDesc &d)
{
    for (int k = 0; k < 3; ++k) {
        d.inv_dx_f[k] = (float)d.inv_dx[k];
        d.ratio_f[k] = (float)(d.inv_dx[k] / d.inv_dx[0]);
    }
    d.div_cx = make_fastdiv((unsigned)d.cells[0]);
    d.div_cy = make_fastdiv((unsigned)d.cells[1]);
}

// Kernel parameter block (passed by value).
struct KParams {
    const SolveDesc *solves;  // device array, tile0 ascending
    int nsolves;
    int use_ctl_dt;           // 1: dt of each solve from its ctl->dt, 0: dt_arg
    int lim_pass;             // k_cfl after the subcell limiter: skip solves with no troubled element
    long long ntiles;         // tiles of this launch (predictor or corrector)
    double dt_arg;
    PdeParams pde;
    Basis b;
    Ops<double> od;
    Ops<float> of;
    // subcell limiter operators (2N+1 subcells): averages of the nodal
    // basis [j][k] and the least-squares reconstruction [k][j]
    double lim_pr[(2 * NMAX - 1) * NMAX];
    double lim_rc[NMAX * (2 * NMAX - 1)];
};

template <typename T> __host__ __device__ inline const Ops<T> &ops_of(const KParams &P);
template <> __host__ __device__ inline const Ops<double> &ops_of<double>(const KParams &P) { return P.od; }
template <> __host__ __device__ inline const Ops<float> &ops_of<float>(const KParams &P) { return P.of; }

__host__ __device__ constexpr int ipow(int b, int e)
{
    int r = 1;
    for (int i = 0; i < e; ++i) r *= b;
    return r;
}
__host__ __device__ constexpr int round_up(int a, int b) { return (a + b - 1) / b * b; }

// ---------------------------------------------------------------------------
// PDE functions.  flux(): all DIM flux components F_d(q) at one point;
// max_eig(): largest |eigenvalue| of dF_d/dQ.
// ---------------------------------------------------------------------------

// The FP32 path works with perturbations about a per-element reference
// state q_ref (held in FP64 in memory): flux_delta returns
// F_d(q_ref + dq) - F_d(q_ref) evaluated from small quantities only, so its
// rounding error scales with |dq| instead of |q|.  Linear systems need no
// reference data (the perturbation flux is the flux of dq).
template <typename T, int M>
struct NoRef {
    T q[M];
};

// 1/x in the compute type, within one ulp (not correctly rounded).  The
// seed is the hardware reciprocal approximation (rcp.approx.ftz: for double
// it reads the leading 32 bits of x, relative error below 2^-19; for float
// about 2^-23), refined by the Newton-Raphson iteration for 1/x, e = 1 - x r,
// r <- r + r e, which squares the relative error, or for double by its
// third-order form r <- r + r (e + e^2), which cubes it (see Muller et al.,
// Handbook of Floating-Point Arithmetic, ch. on Newton-Raphson division).
// Double: 3 FMAs on the FP64 pipe; float: 2 FFMAs.  x is a normal, finite,
// nonzero number wherever the kernels take a reciprocal (densities, volume
// fractions); its result is tested against 1/x (aderdg_device_recip).
#ifdef __CUDACC__
__device__ __forceinline__ double recip(double x)
{
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
    const double e = fma(-x, r, 1.0);
    return fma(r, fma(e, e, e), r);
}
__device__ __forceinline__ float recip(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return fmaf(r, fmaf(-x, r, 1.0f), r);
}
#else
inline double recip(double x) { return 1.0 / x; }
inline float recip(float x) { return 1.0f / x; }
#endif

// Every PDE states: M variables, of which the leading MEV evolve (the rest
// obey q_t = 0); NCP: the system is purely non-conservative (F = 0, all
// terms B_d(q) dq/dx_d, see DiffuseElastic); HAS_SRC: an algebraic source
// S(q) that is linear in q.

// Linear advection F_d = a_d u with the reaction source S = -kappa u
// (kappa = 0 unless given).
template <int DIM>
struct Advection {
    static constexpr int M = 1;
    static constexpr int MEV = M;
    static constexpr bool NCP = false, HAS_SRC = true;
    static constexpr int KIND = 1;
    static constexpr int FLUX_FLOPS = DIM + 1;    // per point, all directions (+ the source)
    static constexpr int EIG_FLOPS = 0;
    template <typename T>
    __device__ __forceinline__ static void source(const PdeParams &P, const T *q, T *S) {
        S[0] = pconst<T>(P, 6) * q[0];  // -kappa q
    }
    template <typename T> using Ref = NoRef<T, M>;
    template <typename T>
    __device__ __forceinline__ static void make_ref(const PdeParams &, const T *q, Ref<T> &r) {
        r.q[0] = q[0];
    }
    template <typename T>
    __device__ __forceinline__ static void flux_delta(const PdeParams &P, const Ref<T> &, const T *dq, T (*f)[M]) {
        flux(P, dq, f);
    }
    template <typename T>
    __device__ __forceinline__ static void flux(const PdeParams &P, const T *q, T (*f)[M]) {
#pragma unroll
        for (int d = 0; d < DIM; ++d) f[d][0] = pconst<T>(P, d) * q[0];
    }
    template <typename T>
    __device__ __forceinline__ static T max_eig(const PdeParams &P, const T *, int d) {
        return pconst<T>(P, 3 + d);
    }
};

// Euler equations (Sec. 3.1, eq. euler), ideal gas.
template <int DIM>
struct Euler {
    static constexpr int M = DIM + 2;
    static constexpr int MEV = M;
    static constexpr bool NCP = false, HAS_SRC = false;
    static constexpr int KIND = 2;
    // 1 reciprocal, DIM products for v, DIM FMA + 2 for p, per direction:
    // DIM FMA/products for momentum + 1 add for pressure + 2 for energy
    static constexpr int FLUX_FLOPS = 1 + DIM + 2 * DIM + 3 + DIM * (2 * DIM + 3);
    static constexpr int EIG_FLOPS = 2 * DIM + 8;
    template <typename T>
    struct Ref {
        T q[M];
        T u0[DIM], EP0;  // reference velocity and E + p
    };
    // reference quantities in the compute type (their rounding only enters
    // the perturbation flux multiplied by perturbations)
    template <typename T>
    __device__ __forceinline__ static void make_ref(const PdeParams &P, const T *q, Ref<T> &r) {
#pragma unroll
        for (int v = 0; v < M; ++v) r.q[v] = q[v];
        const T ir = recip(r.q[0]);
        T kin2 = T(0);
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            r.u0[k] = r.q[1 + k] * ir;
            kin2 += r.q[1 + k] * r.u0[k];
        }
        const T p = pconst<T>(P, 0) * (r.q[DIM + 1] - T(0.5) * kin2);
        r.EP0 = r.q[DIM + 1] + p;
    }
    // F(q_ref + dq) - F(q_ref) from the perturbations:
    //   du = (dm - u0 drho) / rho,  u = u0 + du,
    //   dkin = (m0 . du + dm . u) / 2,  dp = (gamma - 1)(dE - dkin),
    //   dF_rho = dm_d,  dF_m_k = m0_k du_d + dm_k u_d + dp [k == d],
    //   dF_E = du_d (E + p) + u0_d (dE + dp).
    template <typename T>
    __device__ __forceinline__ static void flux_delta(const PdeParams &P, const Ref<T> &r, const T *dq, T (*f)[M]) {
        const T gm1 = pconst<T>(P, 0);
        const T ir = recip(r.q[0] + dq[0]);
        T du[DIM], u[DIM];
        T dkin2 = T(0);
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            du[k] = (dq[1 + k] - r.u0[k] * dq[0]) * ir;
            u[k] = r.u0[k] + du[k];
            dkin2 += r.q[1 + k] * du[k] + dq[1 + k] * u[k];
        }
        const T dE = dq[DIM + 1];
        const T dp = gm1 * (dE - T(0.5) * dkin2);
        const T Ep = r.EP0 + (dE + dp);
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            f[d][0] = dq[1 + d];
#pragma unroll
            for (int k = 0; k < DIM; ++k) f[d][1 + k] = r.q[1 + k] * du[d] + dq[1 + k] * u[d] + (k == d ? dp : T(0));
            f[d][DIM + 1] = du[d] * Ep + r.u0[d] * (dE + dp);
        }
    }
    template <typename T>
    __device__ __forceinline__ static void flux(const PdeParams &P, const T *q, T (*f)[M]) {
        const T gm1 = pconst<T>(P, 0);
        const T ir = recip(q[0]);
        T v[DIM];
        T kin = T(0);
#pragma unroll
        for (int k = 0; k < DIM; ++k) { v[k] = q[1 + k] * ir; kin += q[1 + k] * v[k]; }
        const T E = q[DIM + 1];
        const T p = gm1 * (E - T(0.5) * kin);
        const T Ep = E + p;
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            f[d][0] = q[1 + d];
#pragma unroll
            for (int k = 0; k < DIM; ++k) f[d][1 + k] = q[1 + k] * v[d] + (k == d ? p : T(0));
            f[d][DIM + 1] = v[d] * Ep;
        }
    }
    template <typename T>
    __device__ __forceinline__ static T max_eig(const PdeParams &P, const T *q, int d) {
        const T g = pconst<T>(P, 1);
        const T ir = recip(q[0]);
        T kin = T(0);
#pragma unroll
        for (int k = 0; k < DIM; ++k) kin += q[1 + k] * q[1 + k];
        const T p = pconst<T>(P, 0) * (q[DIM + 1] - T(0.5) * kin * ir);
        return fabs(q[1 + d] * ir) + sqrt(g * p * ir);
    }
};

// Velocity-stress linear elasticity (Sec. 3.2 with alpha = 1, constant
// rho, lambda, mu): Q = (sxx, syy, szz, sxy, syz, sxz, u, v, w).
struct Elastic3 {
    static constexpr int M = 9;
    static constexpr int MEV = M;
    static constexpr bool NCP = false, HAS_SRC = false;
    static constexpr int KIND = 3;
    static constexpr int FLUX_FLOPS = 3 * 9;
    static constexpr int EIG_FLOPS = 0;
    template <typename T> using Ref = NoRef<T, M>;
    template <typename T>
    __device__ __forceinline__ static void make_ref(const PdeParams &, const T *q, Ref<T> &r) {
#pragma unroll
        for (int v = 0; v < M; ++v) r.q[v] = q[v];
    }
    template <typename T>
    __device__ __forceinline__ static void flux_delta(const PdeParams &P, const Ref<T> &, const T *dq, T (*f)[M]) {
        flux(P, dq, f);
    }
    template <typename T>
    __device__ __forceinline__ static void flux(const PdeParams &P, const T *q, T (*f)[M]) {
        const T irho = pconst<T>(P, 0);
        const T lam = pconst<T>(P, 1), mu = pconst<T>(P, 2);
        const T l2m = pconst<T>(P, 3);
        const T u = q[6], v = q[7], w = q[8];
        // x
        f[0][0] = -l2m * u; f[0][1] = -lam * u; f[0][2] = -lam * u;
        f[0][3] = -mu * v;  f[0][4] = T(0);     f[0][5] = -mu * w;
        f[0][6] = -q[0] * irho; f[0][7] = -q[3] * irho; f[0][8] = -q[5] * irho;
        // y
        f[1][0] = -lam * v; f[1][1] = -l2m * v; f[1][2] = -lam * v;
        f[1][3] = -mu * u;  f[1][4] = -mu * w;  f[1][5] = T(0);
        f[1][6] = -q[3] * irho; f[1][7] = -q[1] * irho; f[1][8] = -q[4] * irho;
        // z
        f[2][0] = -lam * w; f[2][1] = -lam * w; f[2][2] = -l2m * w;
        f[2][3] = T(0);     f[2][4] = -mu * v;  f[2][5] = -mu * u;
        f[2][6] = -q[5] * irho; f[2][7] = -q[4] * irho; f[2][8] = -q[2] * irho;
    }
    template <typename T>
    __device__ __forceinline__ static T max_eig(const PdeParams &P, const T *, int) {
        return pconst<T>(P, 4);
    }
};

// Diffuse-interface linear elasticity (Sec. 3.2, the seismic example's
// system) in the state Q = (sigma, w = alpha v, alpha, lambda, mu, rho),
// sigma = (xx, yy, zz, xy, yz, xz) in 3D or the plane-strain (xx, yy, xy) in
// 2D; the last four obey q_t = 0.  No flux: the system is
//   sigma_t - E : (1/alpha) grad(w) + E : (w/alpha^2 (x) grad alpha) = 0,
//   w_t - (alpha/rho) div sigma - (1/rho) sigma grad alpha = 0,
// E : G = lambda tr(G) I + mu (G + G^T).  For a derivative vector g = dQ/dx_d,
// with a_i = (g_{w_i} - w_i g_alpha / alpha) / alpha  (the velocity derivative):
//   B_d(q) g |sigma_ij = -(lambda a_d [i == j] + mu (a_i [j == d] + a_j [i == d]))
//   B_d(q) g |w_i      = -(alpha g_{sigma_id} + sigma_id g_alpha) / rho.
// B_d(q) g is linear in the evolved variables for fixed material fields, so
// a time average of it equals it at the time-averaged state.
template <int DIM>
struct DiffuseElastic {
    static constexpr int NSIG = DIM == 3 ? 6 : 3;
    static constexpr int M = NSIG + DIM + 4;
    static constexpr int MEV = NSIG + DIM;
    static constexpr int IA = MEV, IL = MEV + 1, IM = MEV + 2, IR = MEV + 3;  // alpha lambda mu rho
    static constexpr bool NCP = true, HAS_SRC = false;
    static constexpr int KIND = 4;
    // B(q) times the derivatives at one point, all directions: 2
    // reciprocals; per direction the velocity derivative (4 DIM), the stress
    // rows (~3 NSIG) and the momentum rows (4 DIM); the accumulation over
    // directions (2 M per direction after the first)
    static constexpr int FLUX_FLOPS = 2 + DIM * (8 * DIM + 3 * NSIG) + (DIM - 1) * 2 * M;
    static constexpr int EIG_FLOPS = 4;
    template <typename T> using Ref = NoRef<T, M>;
    template <typename T>
    __device__ __forceinline__ static void make_ref(const PdeParams &, const T *q, Ref<T> &r) {
#pragma unroll
        for (int v = 0; v < M; ++v) r.q[v] = q[v];
    }
    // symmetric-tensor index of (i, j) in the state
    __host__ __device__ static constexpr int sig(int i, int j) {
        return i > j ? sig(j, i)
                     : (i == j ? i : (DIM == 2 ? 2 : (i == 0 && j == 1 ? 3 : (i == 1 && j == 2 ? 4 : 5))));
    }
    // out = B_d(q) g for the state q (absolute values) and g = dQ/dx_d (its
    // evolved part; ga = dalpha/dx_d), with the inverses ia = 1/alpha and
    // ir = 1/rho of q precomputed
    template <typename T>
    __device__ __forceinline__ static void bdot(const T *q, T ia, T ir, int d, const T *g, T ga, T *out) {
        T a[DIM];
#pragma unroll
        for (int i = 0; i < DIM; ++i) a[i] = (g[NSIG + i] - q[NSIG + i] * ia * ga) * ia;
        T ad = a[0];
#pragma unroll
        for (int k = 1; k < DIM; ++k) ad = d == k ? a[k] : ad;
        const T lam = q[IL], mu = q[IM], al = q[IA];
#pragma unroll
        for (int i = 0; i < DIM; ++i)
#pragma unroll
            for (int j = i; j < DIM; ++j) {
                T r = -mu * ((j == d ? a[i] : T(0)) + (i == d ? a[j] : T(0)));
                if (i == j) r -= lam * ad;
                out[sig(i, j)] = r;
            }
#pragma unroll
        for (int i = 0; i < DIM; ++i) {
            T gs = g[sig(i, 0)], qs = q[sig(i, 0)];
#pragma unroll
            for (int k = 1; k < DIM; ++k) {
                gs = d == k ? g[sig(i, k)] : gs;
                qs = d == k ? q[sig(i, k)] : qs;
            }
            out[NSIG + i] = -(al * gs + qs * ga) * ir;
        }
#pragma unroll
        for (int v = MEV; v < M; ++v) out[v] = T(0);
    }
    // J = int_0^1 B_d(qL + s dq) ds dq by the three-point Gauss-Legendre rule
    // on [0, 1] (eq. pc.scheme, straight-segment path); dq = qR - qL
    template <typename T>
    __device__ __forceinline__ static void path_jump(const T *qL, const T *dq, int d, T *J) {
        const T h = T(0.3872983346207416885);  // sqrt(3/5) / 2
        const T sg[3] = {T(0.5) - h, T(0.5), T(0.5) + h};
        const T wg[3] = {T(5.0 / 18.0), T(8.0 / 18.0), T(5.0 / 18.0)};
#pragma unroll
        for (int v = 0; v < M; ++v) J[v] = T(0);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            T ps[M], b[M];
#pragma unroll
            for (int v = 0; v < M; ++v) ps[v] = qL[v] + sg[k] * dq[v];
            bdot(ps, recip(ps[IA]), recip(ps[IR]), d, dq, dq[IA], b);
#pragma unroll
            for (int v = 0; v < MEV; ++v) J[v] += wg[k] * b[v];
        }
    }
    template <typename T>
    __device__ __forceinline__ static void flux(const PdeParams &, const T *, T (*f)[M]) {
#pragma unroll
        for (int d = 0; d < DIM; ++d)
#pragma unroll
            for (int v = 0; v < M; ++v) f[d][v] = T(0);
    }
    template <typename T>
    __device__ __forceinline__ static void flux_delta(const PdeParams &P, const Ref<T> &, const T *q, T (*f)[M]) {
        flux(P, q, f);
    }
    template <typename T>
    __device__ __forceinline__ static T max_eig(const PdeParams &, const T *q, int) {
        return sqrt((q[IL] + T(2) * q[IM]) * recip(q[IR]));  // P-wave speed, independent of alpha
    }
};

// Launch geometry of the per-element kernels.  A trace record holds the
// time-averaged state (M), the time-averaged normal flux (M; not for purely
// non-conservative systems), the wave speed and padding to an even size.
template <class PDE, int DIM, int N>
struct Geom {
    static constexpr int n = N + 1;
    static constexpr int M = PDE::M;
    static constexpr int NS = ipow(n, DIM);        // spatial nodes
    static constexpr int NST = NS * n;             // space-time nodes
    static constexpr int NF = ipow(n, DIM - 1);    // nodes per face
    static constexpr int LAM = PDE::NCP ? M : 2 * M;          // wave speed's index in a record
    static constexpr int RS = (LAM + 1 + 1) / 2 * 2;          // record size
    static constexpr int NREC = DIM * 2 * NF;      // records per element
};

// One compiled launch shape of a per-element kernel: CTA size, elements per
// CTA, dynamic shared memory.
struct TileShape {
    void (*kernel)(KParams);
    int threads, epb;
    size_t smem;
};

// Number of compiled shapes of the predictor and the corrector (shape 0 is
// the default).
constexpr int NSHAPE_P = 9;
constexpr int NSHAPE_C = 6;

// Host-visible description of the compiled kernels of one (PDE, d, N,
// precision).  predictor/corrector and their sizes are the shapes in use;
// pshape/cshape list every compiled shape for the autotuner.
struct KernelSet {
    void (*predictor)(KParams);
    int pred_threads, pred_epb;
    size_t pred_smem;
    void (*corrector)(KParams);
    int corr_threads, corr_epb;
    size_t corr_smem;
    void (*cfl)(KParams);
    int nvar, rs, elem_bytes;  // elem_bytes = sizeof(T)
    int flux_flops, eig_flops;  // per point, for the cost model
    int rf;                     // doubles per element of the FP32 reference record (0: none)
    int ncp;                    // 1: purely non-conservative system (no flux in the records)
    int mx;                     // values per node in the predictor's derivative exchange
    // subcell limiter kernels of instances whose subcell arrays fit one CTA's
    // shared memory (NULL otherwise), 128 threads: minmax, detect and fv in
    // the FP64 instance only, couple in both (its own precision's fluxes)
    void (*lim_minmax)(KParams);
    void (*lim_detect)(KParams);
    void (*lim_fv)(KParams);
    void (*lim_couple)(KParams);
    size_t lim_smem;    // k_lim_fv / k_lim_couple (one element per CTA)
    size_t lim_smem_w;  // k_lim_minmax / k_lim_detect (one element per warp)
    // the FP32 path's extremes and detection (FP32 projections, FP64 where
    // a decision is too close to call), in the FP64 instance only
    void (*lim_minmax32)(KParams);
    void (*lim_detect32)(KParams);
    size_t lim_smem_w32;
    // kept subcell data: the state of uploaded subcell averages (their
    // least-squares reconstruction), in the FP64 instance only
    void (*lim_init)(KParams);
    // the extremes kernels of solves that keep subcell data (FP64, FP32 path)
    void (*lim_minmax_keep)(KParams);
    void (*lim_minmax32_keep)(KParams);
    TileShape pshape[NSHAPE_P], pshape_ex[NSHAPE_P], cshape[NSHAPE_C];  // pshape_ex: extrapolation and CERK guesses
    int pred_shape, corr_shape;  // indices of the shapes in use
};

// Copy of ks that launches predictor shape ps (its extrapolation-guess
// variant if ex) and corrector shape cs.
inline KernelSet with_shapes(const KernelSet &ks, int ps, int cs, bool ex = false)
{
    KernelSet k = ks;
    const TileShape &p = ex ? ks.pshape_ex[ps] : ks.pshape[ps], &c = ks.cshape[cs];
    k.predictor = p.kernel; k.pred_threads = p.threads; k.pred_epb = p.epb; k.pred_smem = p.smem;
    k.corrector = c.kernel; k.corr_threads = c.threads; k.corr_epb = c.epb; k.corr_smem = c.smem;
    k.pred_shape = ps;
    k.corr_shape = cs;
    return k;
}

}  // namespace aderdg
