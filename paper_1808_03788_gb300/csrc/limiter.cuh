// A posteriori subcell finite-volume limiter (Sec. 2.3) of the FP64 path.
//
// After the unlimited step has produced a candidate u* (in place of u^n,
// which the step saved to u_prev):
//   k_lim_minmax  extreme subcell averages of u^n per element and variable
//                 (copied from the last detection where u^n is its candidate)
//   k_lim_detect  troubled elements: non-finite values, Euler positivity at
//                 the nodes and in the subcell averages, or a subcell average
//                 of u* outside the relaxed discrete maximum principle
//                 [lo - delta, hi + delta] of u^n over the element and its
//                 2d face neighbours, delta = max(1e-4, 1e-3 (hi - lo));
//                 flags and a compact list of them
//   k_lim_fv      troubled elements: MUSCL-Hancock with minmod slopes and
//                 Rusanov fluxes on (2N+1)^d subcells of u^n (direction by
//                 direction, ghost subcells two deep from the face
//                 neighbours), then least-squares reconstruction
//   k_lim_couple  unlimited elements next to troubled ones: the DG face
//                 flux the corrector applied on the common face is replaced
//                 by the subcell fluxes projected onto the face nodes
// With kept subcell data (a handle created with limiter 2) an element the
// previous step limited takes the subcell averages that step's subcell
// scheme gave it as its subcell data at t^n (k_lim_minmax moves them into
// place), in the bounds, the subcell scheme and the coupling alike; k_cfl
// takes its wave speeds from them, and k_lim_subcell_init builds a state
// from uploaded subcell averages.
// Both sides of a face between a troubled and an unlimited element, and of
// a face between two troubled ones, evaluate its subcell fluxes with the
// same function on the same subcell averages, so the scheme stays
// conservative.  Each CTA owns one element at a time (grid-stride loop);
// a launch covers every solve of its descriptor list that has the limiter
// (u_prev set), one after the other.
// Included by kernels.cuh inside namespace aderdg.
#pragma once

template <class PDE, int DIM, int N>
struct LimCfg {
    static constexpr int n = N + 1, S = 2 * N + 1, M = PDE::M;
    static constexpr int NS = ipow(n, DIM), NSUB = ipow(S, DIM), NF = ipow(n, DIM - 1), NLINE = ipow(S, DIM - 1);
    static constexpr int THREADS = 128;
    // largest intermediate of a sum-factorised projection or reconstruction
    static constexpr int TMP = cmax(cmax(S * ipow(n, DIM - 1), ipow(S, DIM - 1) * n),
                                    DIM == 3 ? cmax(S * S * n, n * n * S) : 0) * M;
    static constexpr int OPS = round_up(2 * S * n, 2);
    static constexpr int GHOST = 2 * DIM * 2 * NLINE * M;  // [d][side][layer][line][v]
    // subcell face fluxes of one direction (non-conservative systems: the
    // fluctuations of the lower and of the upper subcell)
    static constexpr int FACES = (S + 1) * NLINE * M * (PDE::NCP ? 2 : 1);
    // doubles: operators, staged nodes, own averages, a neighbour's averages,
    // ghost layers, increments, two projection buffers, face fluxes
    static constexpr size_t DOUBLES = OPS + round_up(NS * M, 2) + 3 * (size_t)NSUB * M + GHOST + 2 * TMP + FACES;
    static constexpr size_t BYTES = sizeof(double) * DOUBLES;
    // doubles per line of a stored face record, and per troubled element
    static constexpr int FB = PDE::NCP ? 2 * M : M;
    static constexpr size_t FB_SLOT = (size_t)2 * DIM * NLINE * FB;
    static constexpr bool FITS = BYTES <= 227 * 1024;
    static constexpr bool OK = FITS;
};

// One direction of a tensor-product application: LO points before the
// direction (R of them already transformed), HI after it (C untransformed),
// M values per point; each output is one C-term sum, accumulated in j order.
template <int M, int R, int C, int LO, int HI, typename V>
__device__ __forceinline__ void lim_pass(const V *src, V *dst, const V *Op, int tid, int nt)
{
    constexpr int total = LO * R * HI * M;
    for (int i = tid; i < total; i += nt) {
        const int v = i % M, r = i / M, al = r % LO, ad = (r / LO) % R, ah = r / (LO * R);
        const V *x = src + (al + LO * C * ah) * M + v;
        V acc = V(0);
#pragma unroll
        for (int j = 0; j < C; ++j) acc += Op[ad * C + j] * x[j * LO * M];
        dst[i] = acc;
    }
}

// The same pass by lines: each item is one line (al, ah, v) whose C inputs
// are read once and give its R outputs, each the same C-term sum in j order
// as lim_pass (bitwise the same results, fewer loads and index divisions;
// used by the one-warp FP32 teams, where the FMA pipe is not the limit).
template <int M, int R, int C, int LO, int HI, typename V>
__device__ __forceinline__ void lim_pass_lines(const V *src, V *dst, const V *Op, int tid, int nt)
{
    constexpr int lines = LO * HI * M;
    for (int i = tid; i < lines; i += nt) {
        const int v = i % M, r = i / M, al = r % LO, ah = r / LO;
        const V *x = src + (al + LO * C * ah) * M + v;
        V xin[C];
#pragma unroll
        for (int j = 0; j < C; ++j) xin[j] = x[j * LO * M];
        V *y = dst + (al + LO * R * ah) * M + v;
#pragma unroll
        for (int ad = 0; ad < R; ++ad) {
            V acc = V(0);
#pragma unroll
            for (int j = 0; j < C; ++j) acc += Op[ad * C + j] * xin[j];
            y[ad * LO * M] = acc;
        }
    }
}

// out = (Op (x) ... (x) Op) in along the DIM directions, Op an R x C matrix
// in shared memory ([r][c]); in has C points per direction (x fastest,
// M values per point), out R.  The team -- a CTA or one warp -- is the
// threads tid = 0 .. nt-1, all of which call it; sync() joins them.
template <int DIM, int M, int R, int C, typename V, class Sync>
__device__ void lim_tensor_team(const V *in, V *out, V *ta, V *tb, const V *Op, int tid, int nt, Sync sync)
{
    auto pass = [&](auto lo, auto hi, const V *src, V *dst) {
        constexpr int LO = decltype(lo)::value, HI = decltype(hi)::value;
        if constexpr (sizeof(V) == 4) lim_pass_lines<M, R, C, LO, HI>(src, dst, Op, tid, nt);
        else lim_pass<M, R, C, LO, HI>(src, dst, Op, tid, nt);
    };
    using I1 = std::integral_constant<int, 1>;
    using IC = std::integral_constant<int, C>;
    using IR = std::integral_constant<int, R>;
    if constexpr (DIM == 1) {
        pass(I1{}, I1{}, in, out);
        sync();
    } else if constexpr (DIM == 2) {
        pass(I1{}, IC{}, in, ta);
        sync();
        pass(IR{}, I1{}, ta, out);
        sync();
    } else {
        pass(I1{}, std::integral_constant<int, C * C>{}, in, ta);
        sync();
        pass(IR{}, IC{}, ta, tb);
        sync();
        pass(std::integral_constant<int, R * R>{}, I1{}, tb, out);
        sync();
    }
}

template <int DIM, int M, int R, int C>
__device__ void lim_tensor(const double *in, double *out, double *ta, double *tb, const double *Op)
{
    lim_tensor_team<DIM, M, R, C>(in, out, ta, tb, Op, threadIdx.x, blockDim.x, [] { __syncthreads(); });
}

// Order-preserving integer key of a double that is not NaN (-0 and +0 both
// map to 0): x < y exactly when lim_key(x) < lim_key(y).  Extremes and
// bound tests run on the integer pipe with it; the FP64 pipe, this GPU's
// scarce one, carries only the projections and the admissibility tests.
__device__ __forceinline__ long long lim_key(double x)
{
    const long long b = __double_as_longlong(x);
    return b < 0 ? -(b & 0x7fffffffffffffffLL) : b;
}

__device__ __forceinline__ double lim_unkey(long long k)
{
    return k < 0 ? __longlong_as_double((-k) | (long long)0x8000000000000000ULL) : __longlong_as_double(k);
}

template <class PDE>
__device__ __forceinline__ bool lim_admissible(const PdeParams &P, const double *q)
{
    if constexpr (PDE::KIND == 2) {  // Euler: positive density and pressure
        constexpr int D = PDE::M - 2;
        double kin = 0.0;
#pragma unroll
        for (int k = 0; k < D; ++k) kin += q[1 + k] * q[1 + k];
        const double p = pconst<double>(P, 0) * (q[D + 1] - 0.5 * kin / q[0]);
        return q[0] > 0.0 && p > 0.0;
    } else {
        return true;
    }
}

__device__ __forceinline__ double lim_minmod(double a, double b)
{
    if (a * b <= 0.0) return 0.0;
    return fabs(a) < fabs(b) ? a : b;
}

// Subcell flux across the face between cells b and c of a line along d
// (a, b, c, e: four consecutive subcell averages; r = dt / subcell width):
// minmod slopes, half-step evolution of the two face extrapolations along
// d (MUSCL-Hancock), Rusanov flux.  The one routine every face uses.
template <class PDE, int DIM>
__device__ void lim_face(const PdeParams &P, const double *a, const double *b, const double *c, const double *e, int d,
                         double r, double dt, double *F)
{
    constexpr int M = PDE::M;
    double lo[M], hi[M], qp[M], qm[M], fl[DIM][M], fh[DIM][M], Sv[M];
#pragma unroll
    for (int v = 0; v < M; ++v) {
        const double s = lim_minmod(b[v] - a[v], c[v] - b[v]);
        lo[v] = b[v] - 0.5 * s;
        hi[v] = b[v] + 0.5 * s;
    }
    PDE::flux(P, lo, fl);
    PDE::flux(P, hi, fh);
    if constexpr (PDE::HAS_SRC) PDE::source(P, b, Sv);
#pragma unroll
    for (int v = 0; v < M; ++v) {
        double df = fh[0][v] - fl[0][v];
#pragma unroll
        for (int k = 1; k < DIM; ++k) df = d == k ? fh[k][v] - fl[k][v] : df;
        qp[v] = hi[v] - 0.5 * r * df;
        if constexpr (PDE::HAS_SRC) qp[v] += 0.5 * dt * Sv[v];
    }
#pragma unroll
    for (int v = 0; v < M; ++v) {
        const double s = lim_minmod(c[v] - b[v], e[v] - c[v]);
        lo[v] = c[v] - 0.5 * s;
        hi[v] = c[v] + 0.5 * s;
    }
    PDE::flux(P, lo, fl);
    PDE::flux(P, hi, fh);
    if constexpr (PDE::HAS_SRC) PDE::source(P, c, Sv);
#pragma unroll
    for (int v = 0; v < M; ++v) {
        double df = fh[0][v] - fl[0][v];
#pragma unroll
        for (int k = 1; k < DIM; ++k) df = d == k ? fh[k][v] - fl[k][v] : df;
        qm[v] = lo[v] - 0.5 * r * df;
        if constexpr (PDE::HAS_SRC) qm[v] += 0.5 * dt * Sv[v];
    }
    PDE::flux(P, qp, fl);
    PDE::flux(P, qm, fh);
    const double sl = PDE::max_eig(P, qp, d), sr = PDE::max_eig(P, qm, d);
    const double smax = sl > sr ? sl : sr;
#pragma unroll
    for (int v = 0; v < M; ++v) {
        double fsum = fl[0][v] + fh[0][v];
#pragma unroll
        for (int k = 1; k < DIM; ++k) fsum = d == k ? fl[k][v] + fh[k][v] : fsum;
        F[v] = 0.5 * fsum - 0.5 * smax * (qm[v] - qp[v]);
    }
}

// B_d(q) g of a non-conservative system (zero otherwise)
template <class PDE>
__device__ __forceinline__ void lim_bdot(const double *q, int d, const double *g, double *out)
{
    if constexpr (PDE::NCP) {
        PDE::bdot(q, recip(q[PDE::IA]), recip(q[PDE::IR]), d, g, g[PDE::IA], out);
    } else {
#pragma unroll
        for (int v = 0; v < PDE::M; ++v) out[v] = 0.0;
    }
}

// MUSCL-Hancock half-step of subcell b (neighbours a, c along d; r = dt /
// subcell width): minmod slope s, the two face values evolved by
// -(r/2) (F_d(hi) - F_d(lo) + B_d(b) s) + (dt/2) S(b) into qlo / qhi, and
// that change without the source into chc (any output may be null)
template <class PDE, int DIM>
__device__ void lim_half(const PdeParams &P, const double *a, const double *b, const double *c, int d, double r,
                         double dt, double *s, double *qlo, double *qhi, double *chc)
{
    constexpr int M = PDE::M;
    double sl[M], lo[M], hi[M], fl[DIM][M], fh[DIM][M], Bs[M], Sv[M];
#pragma unroll
    for (int v = 0; v < M; ++v) {
        sl[v] = lim_minmod(b[v] - a[v], c[v] - b[v]);
        lo[v] = b[v] - 0.5 * sl[v];
        hi[v] = b[v] + 0.5 * sl[v];
    }
    PDE::flux(P, lo, fl);
    PDE::flux(P, hi, fh);
    if constexpr (PDE::NCP) lim_bdot<PDE>(b, d, sl, Bs);
    if constexpr (PDE::HAS_SRC) PDE::source(P, b, Sv);
#pragma unroll
    for (int v = 0; v < M; ++v) {
        double df = fh[0][v] - fl[0][v];
#pragma unroll
        for (int k = 1; k < DIM; ++k) df = d == k ? fh[k][v] - fl[k][v] : df;
        if constexpr (PDE::NCP) df += Bs[v];
        double ql = lo[v] - 0.5 * r * df, qh = hi[v] - 0.5 * r * df;
        if constexpr (PDE::HAS_SRC) {
            ql += 0.5 * dt * Sv[v];
            qh += 0.5 * dt * Sv[v];
        }
        if (s) s[v] = sl[v];
        if (qlo) qlo[v] = ql;
        if (qhi) qhi[v] = qh;
        if (chc) chc[v] = -0.5 * r * df;
    }
}

// Path-conservative subcell face along d between cells b and c (a, b, c, e
// consecutive): the lower cell receives Fl = -s_max dq/2 + J/2, the upper
// one Fu = -s_max dq/2 - J/2 (s_max dq on the evolved variables only), dq
// and J between the evolved face values qb (upper value of b) and qc
// (lower value of c), which are returned too (any of them may be null)
template <class PDE, int DIM>
__device__ void lim_face_nc(const PdeParams &P, const double *a, const double *b, const double *c, const double *e,
                            int d, double r, double dt, double *Fl, double *Fu, double *qb_out, double *qc_out)
{
    constexpr int M = PDE::M;
    double qb[M], qc[M], dq[M], J[M];
    lim_half<PDE, DIM>(P, a, b, c, d, r, dt, nullptr, nullptr, qb, nullptr);
    lim_half<PDE, DIM>(P, b, c, e, d, r, dt, nullptr, qc, nullptr, nullptr);
#pragma unroll
    for (int v = 0; v < M; ++v) dq[v] = qc[v] - qb[v];
    PDE::path_jump(qb, dq, d, J);
    const double sl = PDE::max_eig(P, qb, d), sr = PDE::max_eig(P, qc, d);
    const double smax = sl > sr ? sl : sr;
#pragma unroll
    for (int v = 0; v < M; ++v) {
        const double f = v < PDE::MEV ? -(0.5 * smax * dq[v]) : 0.0;
        if (Fl) Fl[v] = f + 0.5 * J[v];
        if (Fu) Fu[v] = f - 0.5 * J[v];
        if (qb_out) qb_out[v] = qb[v];
        if (qc_out) qc_out[v] = qc[v];
    }
}

// index of the subcell at position i along d on line l (the other indices
// of l in increasing direction order)
template <int DIM, int S>
__device__ __forceinline__ int lim_cell(int d, int l, int i)
{
    int idx = 0, pw = 1, rem = l;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        int x;
        if (k == d) {
            x = i;
        } else {
            x = rem % S;
            rem /= S;
        }
        idx += x * pw;
        pw *= S;
    }
    return idx;
}

// Shared-memory layout of the limiter kernels.
template <class L>
struct LimSmem {
    double *Pr, *Rc, *u, *avg, *nb, *ghost, *dq, *ta, *tb, *fb;
    __device__ explicit LimSmem(double *base)
    {
        Pr = base;
        Rc = Pr + L::S * L::n;
        u = base + L::OPS;
        avg = u + round_up(L::NS * L::M, 2);
        nb = avg + (size_t)L::NSUB * L::M;
        ghost = nb + (size_t)L::NSUB * L::M;
        dq = ghost + L::GHOST;
        ta = dq + (size_t)L::NSUB * L::M;
        tb = ta + L::TMP;
        fb = tb + L::TMP;
    }
};

// whether a limited solve of the launch has a troubled element this step
// (the subcell scheme and the coupling have nothing to do otherwise)
__device__ __forceinline__ bool lim_any_troubled(const KParams &P)
{
    for (int si = 0; si < P.nsolves; ++si) {
        const SolveDesc &S = P.solves[si];
        if (S.u_prev && S.ctl->lim_count != 0u) return true;
    }
    return false;
}

template <class L>
__device__ void lim_load_ops(const KParams &P, LimSmem<L> &sm)
{
    for (int i = threadIdx.x; i < L::S * L::n; i += blockDim.x) {
        sm.Pr[i] = P.lim_pr[i];
        sm.Rc[i] = P.lim_rc[i];
    }
    __syncthreads();
}

// subcell averages of element e's nodal state src into dst
template <class L, int DIM>
__device__ void lim_averages(const double *src, long long e, LimSmem<L> &sm, double *dst)
{
    for (int i = threadIdx.x; i < L::NS * L::M; i += blockDim.x) sm.u[i] = src[e * (L::NS * L::M) + i];
    __syncthreads();
    lim_tensor<DIM, L::M, L::S, L::n>(sm.u, dst, sm.ta, sm.tb, sm.Pr);
}

// Subcell data of element e at t^n (eq. subcellaverage): where the solve
// keeps subcell data and lim_kept[e] is set (the step that produced u^n
// limited e), the averages that step's subcell scheme gave it; else the
// averages of its nodal state u_prev.  The CTA works on one element.
template <class L, int DIM>
__device__ void lim_un_averages(const SolveDesc &S, long long e, LimSmem<L> &sm, double *dst)
{
    if (S.lim_sub && S.lim_kept[e]) {  // uniform over the CTA
        const double *src = S.lim_sub + e * (L::NSUB * L::M);
        for (int i = threadIdx.x; i < L::NSUB * L::M; i += blockDim.x) dst[i] = src[i];
        __syncthreads();
    } else {
        lim_averages<L, DIM>(S.u_prev, e, sm, dst);
    }
}

// the two subcell layers of averages a next to face (d, side) into
// ghost slot g[layer][line][v]: side 0 -> layers 0, 1; side 1 -> S-2, S-1
template <class L, int DIM>
__device__ void lim_layers(const double *a, int d, int side, double *g)
{
    for (int i = threadIdx.x; i < 2 * L::NLINE * L::M; i += blockDim.x) {
        const int v = i % L::M, r = i / L::M, l = r % L::NLINE, layer = r / L::NLINE;
        const int pos = side ? L::S - 2 + layer : layer;
        g[i] = a[lim_cell<DIM, L::S>(d, l, pos) * L::M + v];
    }
}

// Per-warp shared memory of the element-per-warp kernels (minmax, detect):
// staged nodes, subcell averages, two projection buffers.
template <class L>
struct LimWarp {
    static constexpr size_t DOUBLES = round_up(L::NS * L::M, 2) + (size_t)L::NSUB * L::M + 2 * L::TMP;
    static constexpr int WARPS = cmax(1, cmin(4, (int)((200 * 1024) / (8 * DOUBLES))));
    static constexpr size_t BYTES = sizeof(double) * (round_up(2 * L::S * L::n, 2) + WARPS * DOUBLES);
};

// subcell averages of element e's nodal state src, by one warp into avg
template <class L, int DIM>
__device__ void lim_averages_warp(const double *src, long long e, const double *Pr, double *u, double *avg, double *ta,
                                  double *tb, int lane)
{
    for (int i = lane; i < L::NS * L::M; i += 32) u[i] = src[e * (L::NS * L::M) + i];
    __syncwarp();
    lim_tensor_team<DIM, L::M, L::S, L::n>(u, avg, ta, tb, Pr, lane, 32, [] { __syncwarp(); });
}

// extreme subcell averages of one element (warp-wide), written to
// mm[v][lo, hi]; the same routine for u^n and for the candidate, so that a
// candidate's extremes can stand for the next step's u^n bit for bit
template <class L>
__device__ void lim_extremes_warp(const double *avg, int lane, double *mm)
{
    for (int v = 0; v < L::M; ++v) {
        long long lo = lim_key(avg[v]), hi = lo;
        for (int a = lane; a < L::NSUB; a += 32) {
            const long long k = lim_key(avg[a * L::M + v]);
            lo = k < lo ? k : lo;
            hi = k > hi ? k : hi;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const long long ol = __shfl_xor_sync(0xffffffffu, lo, o), oh = __shfl_xor_sync(0xffffffffu, hi, o);
            lo = ol < lo ? ol : lo;
            hi = oh > hi ? oh : hi;
        }
        if (lane == 0) {
            mm[v * 2] = lim_unkey(lo);
            mm[v * 2 + 1] = lim_unkey(hi);
        }
    }
}

// Kept subcell data: element e's averages from the last limited step
// (lim_subn) become its subcell data of u^n (lim_sub) and give its extremes
// (the same set of values as lim_extremes_warp takes, so the same extremes).
// One warp; lane l takes subcells l, l + 32, ..., their loads issued in
// groups of up to four subcells before any is used (one memory round trip
// per group, not one per value).  Out of line, so that the kept elements do
// not weigh on the registers of the extremes kernels' common path.
template <class L>
__device__ __noinline__ void lim_move_kept(const SolveDesc &S, long long e, int lane)
{
    constexpr int M = L::M, NSUB = L::NSUB, PER = (NSUB + 31) / 32, CH = PER < 4 ? PER : 4;
    const double *src = S.lim_subn + e * (NSUB * M);
    double *dst = S.lim_sub + e * (NSUB * M);
    long long lo[M], hi[M];
#pragma unroll
    for (int v = 0; v < M; ++v) {
        lo[v] = 0x7fffffffffffffffll;
        hi[v] = -0x7fffffffffffffffll - 1;
    }
#pragma unroll 1
    for (int r0 = 0; r0 < PER; r0 += CH) {
        double x[CH][M];
#pragma unroll
        for (int r = 0; r < CH; ++r) {
            const int a = lane + 32 * (r0 + r);
            if (r0 + r < PER && a < NSUB) {
#pragma unroll
                for (int v = 0; v < M; ++v) x[r][v] = src[a * M + v];
            }
        }
#pragma unroll
        for (int r = 0; r < CH; ++r) {
            const int a = lane + 32 * (r0 + r);
            if (r0 + r < PER && a < NSUB) {
#pragma unroll
                for (int v = 0; v < M; ++v) {
                    dst[a * M + v] = x[r][v];
                    const long long k = lim_key(x[r][v]);
                    lo[v] = k < lo[v] ? k : lo[v];
                    hi[v] = k > hi[v] ? k : hi[v];
                }
            }
        }
    }
#pragma unroll
    for (int v = 0; v < M; ++v) {
        long long l = lo[v], h = hi[v];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const long long ol = __shfl_xor_sync(0xffffffffu, l, o), oh = __shfl_xor_sync(0xffffffffu, h, o);
            l = ol < l ? ol : l;
            h = oh > h ? oh : h;
        }
        if (lane == 0) {
            S.lim_mm[e * (2 * M) + v * 2] = lim_unkey(l);
            S.lim_mm[e * (2 * M) + v * 2 + 1] = lim_unkey(h);
        }
    }
}

// Extremes of u^n.  After a limited step on the same state (ctl->lim_fresh),
// an element that was not troubled and had no troubled face neighbour
// still holds the candidate the detection projected, so its extremes are
// copied from there; the others (and all after a state upload or an
// explicit corrector call) are projected afresh.  Where the solve keeps
// subcell data (ctl->lim_kept_ok), an element the last limited step
// treated takes the subcell averages that step gave it (lim_subn) as its
// subcell data at t^n: they move to lim_sub, lim_kept[e] is set, and they
// give its extremes; lim_kept is cleared for every other element.  KEEP:
// the instance for solves that keep subcell data (the other one is the
// plain limiter's, without that path).
template <class PDE, int DIM, int N, bool KEEP>
__global__ void __launch_bounds__(128) k_lim_minmax(const KParams P)
{
    using L = LimCfg<PDE, DIM, N>;
    using W = LimWarp<L>;
    if constexpr (L::OK) {
        extern __shared__ __align__(16) unsigned char smem_raw[];
        double *Pr = reinterpret_cast<double *>(smem_raw);
        for (int i = threadIdx.x; i < L::S * L::n; i += blockDim.x) Pr[i] = P.lim_pr[i];
        __syncthreads();
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        if (warp >= W::WARPS) return;
        double *u = Pr + round_up(2 * L::S * L::n, 2) + warp * W::DOUBLES;
        double *avg = u + round_up(L::NS * L::M, 2), *ta = avg + (size_t)L::NSUB * L::M, *tb = ta + L::TMP;
        for (int si = 0; si < P.nsolves; ++si) {
            const SolveDesc &S = P.solves[si];
            if (!S.u_prev) continue;  // a solve without the limiter
            const bool fresh = S.ctl->lim_fresh != 0;
            const bool kept_ok = KEEP && S.lim_sub && S.ctl->lim_kept_ok != 0;
            for (long long e = (long long)blockIdx.x * W::WARPS + warp; e < S.E; e += (long long)gridDim.x * W::WARPS) {
                if constexpr (KEEP) {
                    if (S.lim_sub) {
                        const int kept = kept_ok && S.lim_flags[e] != 0;
                        if (lane == 0) S.lim_kept[e] = kept;
                        if (kept) {  // uniform over the warp
                            lim_move_kept<L>(S, e, lane);
                            continue;
                        }
                    }
                }
                bool reuse = fresh;
                if (reuse) {
                    int touched = S.lim_flags[e];
#pragma unroll
                    for (int d = 0; d < DIM; ++d)
#pragma unroll
                        for (int side = 0; side < 2; ++side)
                            touched |=
                                S.lim_flags[neighbour_of(S, (int)e, d, side ? 1 : -1)];
                    reuse = !touched;
                }
                if (reuse) {  // uniform over the warp
                    if (lane < 2 * L::M) S.lim_mm[e * (2 * L::M) + lane] = S.lim_mmc[e * (2 * L::M) + lane];
                    continue;
                }
                lim_averages_warp<L, DIM>(S.u_prev, e, Pr, u, avg, ta, tb, lane);
                lim_extremes_warp<L>(avg, lane, S.lim_mm + e * (2 * L::M));
                __syncwarp();
            }
        }
    }
}

template <class PDE, int DIM, int N>
__global__ void __launch_bounds__(128) k_lim_detect(const KParams P)
{
    using L = LimCfg<PDE, DIM, N>;
    using W = LimWarp<L>;
    if constexpr (L::OK) {
        extern __shared__ __align__(16) unsigned char smem_raw[];
        double *Pr = reinterpret_cast<double *>(smem_raw);
        for (int i = threadIdx.x; i < L::S * L::n; i += blockDim.x) Pr[i] = P.lim_pr[i];
        __syncthreads();
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        if (warp >= W::WARPS) return;
        double *u = Pr + round_up(2 * L::S * L::n, 2) + warp * W::DOUBLES;
        double *avg = u + round_up(L::NS * L::M, 2), *ta = avg + (size_t)L::NSUB * L::M, *tb = ta + L::TMP;
        for (int si = 0; si < P.nsolves; ++si) {
            const SolveDesc &S = P.solves[si];
            if (!S.u_prev) continue;
            // this launch keeps the candidate's extremes for the next step
            // (and, with kept subcell data, the subcell scheme of this step
            // leaves the troubled elements' averages in lim_subn)
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                S.ctl->lim_fresh = 1u;
                S.ctl->lim_kept_ok = 1u;
            }
            for (long long e = (long long)blockIdx.x * W::WARPS + warp; e < S.E; e += (long long)gridDim.x * W::WARPS) {
                const double *uc = S.u_out + e * (L::NS * L::M);  // the candidate
                int bad = 0;
                for (int s = lane; s < L::NS; s += 32) {
                    double q[L::M];
                    bool fin = true;
#pragma unroll
                    for (int v = 0; v < L::M; ++v) {
                        q[v] = uc[s * L::M + v];
                        fin = fin && !dbl_nonfinite(q[v]);
                    }
                    bad |= !fin || !lim_admissible<PDE>(P.pde, q);
                }
                bad = __any_sync(0xffffffffu, bad);
                if (!bad) {
                    lim_averages_warp<L, DIM>(S.u_out, e, Pr, u, avg, ta, tb, lane);
                    // the candidate's extremes, the next step's u^n extremes if
                    // this element stays untouched
                    lim_extremes_warp<L>(avg, lane, S.lim_mmc + e * (2 * L::M));
                    for (int a = lane; a < L::NSUB; a += 32) bad |= !lim_admissible<PDE>(P.pde, avg + a * L::M);
                    for (int v = 0; v < L::M; ++v) {
                        // the relaxed maximum principle of u^n over the element and its face neighbours
                        long long klo = lim_key(S.lim_mm[(e * L::M + v) * 2]);
                        long long khi = lim_key(S.lim_mm[(e * L::M + v) * 2 + 1]);
#pragma unroll
                        for (int d = 0; d < DIM; ++d)
#pragma unroll
                            for (int side = 0; side < 2; ++side) {
                                const long long nb =
                                    neighbour_of(S, (int)e, d, side ? 1 : -1);
                                const long long kl = lim_key(S.lim_mm[(nb * L::M + v) * 2]);
                                const long long kh = lim_key(S.lim_mm[(nb * L::M + v) * 2 + 1]);
                                klo = kl < klo ? kl : klo;
                                khi = kh > khi ? kh : khi;
                            }
                        const double lo = lim_unkey(klo), hi = lim_unkey(khi);
                        const double delta = fmax(1e-4, 1e-3 * (hi - lo));
                        const long long blo = lim_key(lo - delta), bhi = lim_key(hi + delta);
                        for (int a = lane; a < L::NSUB; a += 32) {
                            const long long k = lim_key(avg[a * L::M + v]);
                            bad |= k < blo || k > bhi;
                        }
                    }
                    bad = __any_sync(0xffffffffu, bad);
                }
                if (lane == 0) {
                    S.lim_flags[e] = bad;
                    if (bad) {
                        // at most E entries a step (the reset after the limiter empties it)
                        const unsigned k = atomicAdd(&S.ctl->lim_count, 1u);
                        if (k < (unsigned)S.E) {
                            S.lim_list[k] = (int)e;
                            if (S.lim_slot) S.lim_slot[e] = (int)k;
                        }
                    }
                }
                __syncwarp();
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Detection on the FP32 path (Sec. 2.3).  The subcell averages are projected
// in FP32 from the perturbations dq = u - u_ref of the element's nodes
// (u_ref: its first node, in FP64), so that their rounding scales with the
// element's variation, not with the state.  Every decision that an FP32
// value is too close to call is taken again in FP64: a subcell average within
// the error bound of a maximum-principle bound is recomputed from the FP64
// nodes and compared with the FP64 bound, and an Euler subcell whose FP32
// density or pressure is within its error bound of zero has its averages
// recomputed in FP64 and tested exactly.  The error bound of an average of
// variable v is TOLC eps32 rho^d max_s |dq_sv| (rho = the largest absolute
// row sum of the projection; TOLC covers the d passes of n-term sums, the
// narrowing of dq and of the operator, with a factor 2 to spare), plus eps32
// times the bound itself.  The extremes the detection keeps for the next
// step (and the ones k_lim_minmax32 computes) are u_ref plus the FP32
// extremes, the same routine for the state and for the candidate.
// ---------------------------------------------------------------------------
template <class L>
struct LimWarp32 {
    // floats per warp: node perturbations, subcell averages, two projection buffers
    static constexpr size_t FLOATS =
        (size_t)round_up(L::NS * L::M, 4) + round_up(L::NSUB * L::M, 4) + 2 * (size_t)round_up(L::TMP, 4);
    static constexpr int WARPS = cmax(1, cmin(4, (int)((200 * 1024) / (4 * FLOATS))));
    static constexpr int PR64 = round_up(L::S * L::n, 2);  // doubles: the FP64 operator (rechecks)
    static constexpr int PR32 = round_up(L::S * L::n, 4);  // floats: the FP32 operator
    static constexpr size_t BYTES = 8 * (size_t)PR64 + 4 * (size_t)PR32 + 4 * WARPS * FLOATS;
    static constexpr float TOLC = 2.0f * (L::n + 2) * 3 + 8.0f;  // d (n + 2) + 4, doubled, for d <= 3
    static_assert(round_up(L::TMP, 4) >= 4 * L::M, "the detection keeps 2 M doubles of bounds in ta");
};

// The FP64 subcell average a of variable v from the FP64 nodes x of one
// element (one lane; the tensor sums of the projection, innermost x).
template <class L, int DIM>
__device__ double lim_average64(const double *x, const double *Pr, int a, int v)
{
    constexpr int n = L::n, S = L::S, M = L::M;
    const int ax = a % S, ay = (a / S) % S, az = a / (S * S);
    double acc = 0.0;
    for (int jz = 0; jz < (DIM == 3 ? n : 1); ++jz) {
        double accy = 0.0;
        for (int jy = 0; jy < n; ++jy) {
            double accx = 0.0;
            for (int jx = 0; jx < n; ++jx) accx += Pr[ax * n + jx] * x[((jz * n + jy) * n + jx) * M + v];
            accy += Pr[ay * n + jy] * accx;
        }
        acc = DIM == 3 ? acc + Pr[az * n + jz] * accy : accy;
    }
    return acc;
}

// FP32 subcell averages of element e of src (warp-wide): ref = its first
// node (every lane), u = narrowed perturbations, avg = their averages; lane
// v < M also gets its variable's reference ref_l and largest perturbation
// am_l (the per-variable FP64 work then runs once per warp instruction,
// one variable per lane).
template <class L, int DIM>
__device__ __forceinline__ void lim_averages32_warp(const double *src, long long e, const float *Pr32, float *u, float *avg,
                                                    float *ta, float *tb, int lane, double *ref, double &ref_l,
                                                    float &am_l)
{
    constexpr int M = L::M;
    const double *x = src + e * (L::NS * M);
    float am[M];
#pragma unroll
    for (int v = 0; v < M; ++v) {
        ref[v] = x[v];
        am[v] = 0.f;
    }
    for (int s = lane; s < L::NS; s += 32) {
#pragma unroll
        for (int v = 0; v < M; ++v) {
            const float d = dbl_to_flt_rn(x[s * M + v] - ref[v]);
            u[s * M + v] = d;
            am[v] = fmaxf(am[v], fabsf(d));
        }
    }
    ref_l = 0.0;
    am_l = 0.f;
#pragma unroll
    for (int v = 0; v < M; ++v) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) am[v] = fmaxf(am[v], __shfl_xor_sync(0xffffffffu, am[v], o));
        am_l = lane == v ? am[v] : am_l;
        ref_l = lane == v ? ref[v] : ref_l;
    }
    __syncwarp();
    lim_tensor_team<DIM, M, L::S, L::n>(u, avg, ta, tb, Pr32, lane, 32, [] { __syncwarp(); });
}

// Extremes of the FP32 averages (warp-wide), kept as ref + widened value;
// lane v < M writes variable v's pair.
template <class L>
__device__ __forceinline__ void lim_extremes32_warp(const float *avg, double ref_l, int lane, double *mm)
{
    float lo[L::M], hi[L::M];
    NodeIO<float, L::M>::load(avg, lo);  // subcell 0 seeds every lane
#pragma unroll
    for (int v = 0; v < L::M; ++v) hi[v] = lo[v];
    for (int a = lane; a < L::NSUB; a += 32) {  // each subcell's averages in one vector read
        float x[L::M];
        NodeIO<float, L::M>::load(avg + a * L::M, x);
#pragma unroll
        for (int v = 0; v < L::M; ++v) {
            lo[v] = fminf(lo[v], x[v]);
            hi[v] = fmaxf(hi[v], x[v]);
        }
    }
    float lo_l = 0.f, hi_l = 0.f;
#pragma unroll
    for (int v = 0; v < L::M; ++v) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo[v] = fminf(lo[v], __shfl_xor_sync(0xffffffffu, lo[v], o));
            hi[v] = fmaxf(hi[v], __shfl_xor_sync(0xffffffffu, hi[v], o));
        }
        lo_l = lane == v ? lo[v] : lo_l;
        hi_l = lane == v ? hi[v] : hi_l;
    }
    if (lane < L::M) {
        mm[lane * 2] = ref_l + flt_to_dbl(lo_l);
        mm[lane * 2 + 1] = ref_l + flt_to_dbl(hi_l);
    }
}

// Shared layout of the FP32-path kernels: FP64 operator, FP32 operator,
// then per warp its buffers; returns this warp's first buffer, sets rhoD.
template <class L, int DIM>
__device__ __forceinline__ float *lim32_setup(const KParams &P, unsigned char *smem, double **Pr64, float **Pr32, float *rhoD)
{
    using W = LimWarp32<L>;
    double *p64 = reinterpret_cast<double *>(smem);
    float *p32 = reinterpret_cast<float *>(p64 + W::PR64);
    for (int i = threadIdx.x; i < L::S * L::n; i += blockDim.x) {
        p64[i] = P.lim_pr[i];
        p32[i] = dbl_to_flt_rn(P.lim_pr[i]);
    }
    __syncthreads();
    float rho = 0.f;
    for (int a = 0; a < L::S; ++a) {
        float r = 0.f;
        for (int j = 0; j < L::n; ++j) r += fabsf(p32[a * L::n + j]);
        rho = fmaxf(rho, r);
    }
    float rd = 1.f;
    for (int d = 0; d < DIM; ++d) rd *= rho * 1.001f;
    *rhoD = rd;
    *Pr64 = p64;
    *Pr32 = p32;
    return p32 + W::PR32 + (size_t)(threadIdx.x >> 5) * W::FLOATS;
}

// Extremes of u^n on the FP32 path (as k_lim_minmax, FP32 projections;
// KEEP as there).
template <class PDE, int DIM, int N, bool KEEP>
__global__ void __launch_bounds__(128) k_lim_minmax32(const KParams P)
{
    using L = LimCfg<PDE, DIM, N>;
    using W = LimWarp32<L>;
    if constexpr (L::OK) {
        extern __shared__ __align__(16) unsigned char smem_raw[];
        double *Pr64;
        float *Pr32, rhoD;
        float *u = lim32_setup<L, DIM>(P, smem_raw, &Pr64, &Pr32, &rhoD);
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        if (warp >= W::WARPS) return;
        float *avg = u + round_up(L::NS * L::M, 4), *ta = avg + round_up(L::NSUB * L::M, 4),
              *tb = ta + round_up(L::TMP, 4);
        for (int si = 0; si < P.nsolves; ++si) {
            const SolveDesc &S = P.solves[si];
            if (!S.u_prev) continue;  // a solve without the limiter
            const bool fresh = S.ctl->lim_fresh != 0;
            const bool kept_ok = KEEP && S.lim_sub && S.ctl->lim_kept_ok != 0;
            // 32 elements per warp at a time: each lane decides for its own
            // element and copies the kept extremes; the warp then projects
            // the elements that need it (or moves their kept subcell data,
            // as k_lim_minmax does), one after the other
            for (long long e0 = ((long long)blockIdx.x * W::WARPS + warp) * 32; e0 < S.E;
                 e0 += (long long)gridDim.x * W::WARPS * 32) {
                const long long el = e0 + lane;
                bool need = el < S.E, kept = false;
                unsigned kmask = 0u;
                if constexpr (KEEP) {
                    if (need && S.lim_sub) {
                        kept = kept_ok && S.lim_flags[el] != 0;
                        S.lim_kept[el] = kept;
                    }
                    kmask = __ballot_sync(0xffffffffu, kept);
                }
                if (need && fresh && !kept) {
                    int touched = S.lim_flags[el];
#pragma unroll
                    for (int d = 0; d < DIM; ++d)
#pragma unroll
                        for (int side = 0; side < 2; ++side)
                            touched |=
                                S.lim_flags[neighbour_of(S, (int)el, d, side ? 1 : -1)];
                    if (!touched) {
#pragma unroll
                        for (int k = 0; k < 2 * L::M; ++k) S.lim_mm[el * (2 * L::M) + k] = S.lim_mmc[el * (2 * L::M) + k];
                        need = false;
                    }
                }
                unsigned todo = __ballot_sync(0xffffffffu, need);
                while (todo) {  // uniform over the warp
                    const int j = __ffs(todo) - 1;
                    const long long e = e0 + j;
                    todo &= todo - 1;
                    if constexpr (KEEP) {
                        if ((kmask >> j) & 1u) {
                            lim_move_kept<L>(S, e, lane);
                            continue;
                        }
                    }
                    double ref[L::M], ref_l;
                    float am_l;
                    lim_averages32_warp<L, DIM>(S.u_prev, e, Pr32, u, avg, ta, tb, lane, ref, ref_l, am_l);
                    lim_extremes32_warp<L>(avg, ref_l, lane, S.lim_mm + e * (2 * L::M));
                    __syncwarp();
                }
            }
        }
    }
}

// Euler admissibility of one FP32 subcell average (absolute state refF +
// avg, refF the element's reference rounded to float once): 1 admissible,
// 0 not, -1 too close to call in FP32.
template <class PDE>
__device__ __forceinline__ int lim_admissible32(const PdeParams &P, const float *refF, const float *avg)
{
    if constexpr (PDE::KIND == 2) {
        constexpr int D = PDE::M - 2;
        float q[PDE::M];
        float mag = 0.f;
#pragma unroll
        for (int v = 0; v < PDE::M; ++v) {
            q[v] = refF[v] + avg[v];
            mag = fmaxf(mag, fabsf(q[v]));
        }
        if (q[0] <= 1e-6f * mag) return q[0] < -1e-6f * mag ? 0 : -1;
        float kin = 0.f;
#pragma unroll
        for (int k = 0; k < D; ++k) kin += q[1 + k] * q[1 + k];
        const float e2 = 0.5f * kin * recip(q[0]);  // within 1 ulp: far inside the 1e-5 band
        const float p = pconst<float>(P, 0) * (q[D + 1] - e2);
        const float err = 1e-5f * (fabsf(q[D + 1]) + e2) * pconst<float>(P, 0);
        return p > err ? 1 : (p < -err ? 0 : -1);
    } else {
        return 1;
    }
}

template <class PDE, int DIM, int N>
__global__ void __launch_bounds__(128) k_lim_detect32(const KParams P)
{
    using L = LimCfg<PDE, DIM, N>;
    using W = LimWarp32<L>;
    if constexpr (L::OK) {
        extern __shared__ __align__(16) unsigned char smem_raw[];
        double *Pr64;
        float *Pr32, rhoD;
        float *u = lim32_setup<L, DIM>(P, smem_raw, &Pr64, &Pr32, &rhoD);
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        if (warp >= W::WARPS) return;
        float *avg = u + round_up(L::NS * L::M, 4), *ta = avg + round_up(L::NSUB * L::M, 4),
              *tb = ta + round_up(L::TMP, 4);
        constexpr float EPS = 5.9604645e-08f;  // 2^-24
        for (int si = 0; si < P.nsolves; ++si) {
            const SolveDesc &S = P.solves[si];
            if (!S.u_prev) continue;
            // this launch keeps the candidate's extremes for the next step
            // (and, with kept subcell data, the subcell scheme of this step
            // leaves the troubled elements' averages in lim_subn)
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                S.ctl->lim_fresh = 1u;
                S.ctl->lim_kept_ok = 1u;
            }
            for (long long e = (long long)blockIdx.x * W::WARPS + warp; e < S.E; e += (long long)gridDim.x * W::WARPS) {
                const double *uc = S.u_out + e * (L::NS * L::M);  // the candidate
                int bad = 0;
                for (int s = lane; s < L::NS; s += 32) {
                    bool fin = true;
#pragma unroll
                    for (int v = 0; v < L::M; ++v) fin = fin && !dbl_nonfinite(uc[s * L::M + v]);
                    bad |= !fin;
                }
                bad = __any_sync(0xffffffffu, bad);
                if (!bad) {
                    double ref[L::M], ref_l;
                    float am_l;
                    lim_averages32_warp<L, DIM>(S.u_out, e, Pr32, u, avg, ta, tb, lane, ref, ref_l, am_l);
                    lim_extremes32_warp<L>(avg, ref_l, lane, S.lim_mmc + e * (2 * L::M));
                    // admissibility at the nodes: FP32 on ref + perturbation, FP64
                    // where that is too close to call
                    float refF[L::M];
#pragma unroll
                    for (int v = 0; v < L::M; ++v) refF[v] = PDE::KIND == 2 ? dbl_to_flt_rn(ref[v]) : 0.f;
                    for (int s = lane; s < L::NS; s += 32) {
                        int ok = lim_admissible32<PDE>(P.pde, refF, u + s * L::M);
                        if (ok < 0) ok = lim_admissible<PDE>(P.pde, uc + s * L::M) ? 1 : 0;
                        bad |= ok == 0;
                    }
                    for (int a = lane; a < L::NSUB; a += 32) {
                        int ok = lim_admissible32<PDE>(P.pde, refF, avg + a * L::M);
                        if (ok < 0) {  // too close to call: the subcell's FP64 averages
                            double q[L::M];
#pragma unroll
                            for (int v = 0; v < L::M; ++v) q[v] = lim_average64<L, DIM>(uc, Pr64, a, v);
                            ok = lim_admissible<PDE>(P.pde, q) ? 1 : 0;
                        }
                        bad |= ok == 0;
                    }
                    // the relaxed maximum principle of u^n over the element and
                    // its face neighbours: lane v forms variable v's bounds
                    double lo_l = 0.0, hi_l = 0.0;
                    float rlo_l = 0.f, rhi_l = 0.f, tol_l = 0.f;
                    if (lane < L::M) {
                        const int v = lane;
                        long long klo = lim_key(S.lim_mm[(e * L::M + v) * 2]);
                        long long khi = lim_key(S.lim_mm[(e * L::M + v) * 2 + 1]);
#pragma unroll
                        for (int d = 0; d < DIM; ++d)
#pragma unroll
                            for (int side = 0; side < 2; ++side) {
                                const long long nb =
                                    neighbour_of(S, (int)e, d, side ? 1 : -1);
                                const long long kl = lim_key(S.lim_mm[(nb * L::M + v) * 2]);
                                const long long kh = lim_key(S.lim_mm[(nb * L::M + v) * 2 + 1]);
                                klo = kl < klo ? kl : klo;
                                khi = kh > khi ? kh : khi;
                            }
                        lo_l = lim_unkey(klo);
                        hi_l = lim_unkey(khi);
                        // the relaxed bounds lo - delta, hi + delta in FP32 about
                        // the reference (two FP64 differences): dlo, dhi are
                        // within eps/2 of exact, delta within a few eps of
                        // delta, and the band below takes 6 eps of the
                        // bounds' magnitude for these roundings
                        const float dlo = dbl_to_flt_rn(lo_l - ref_l), dhi = dbl_to_flt_rn(hi_l - ref_l);
                        const float delta = fmaxf(1e-4f, 1e-3f * (dhi - dlo));
                        rlo_l = dlo - delta;
                        rhi_l = dhi + delta;
                        tol_l = W::TOLC * EPS * rhoD * am_l + 6.f * EPS * fmaxf(fabsf(rlo_l), fabsf(rhi_l)) + 1e-30f;
                    }
                    // every lane gets all variables' FP32 bands [lo - tol, lo + tol]
                    // and [hi - tol, hi + tol] around the bounds; each subcell's
                    // averages are read once.  The FP64 bounds, for the rare
                    // rechecks, wait in the projection buffer ta (free by now).
                    double *bnd = reinterpret_cast<double *>(ta);
                    if (lane < L::M) {
                        bnd[2 * lane] = lo_l;
                        bnd[2 * lane + 1] = hi_l;
                    }
                    __syncwarp();
                    // the FP64 bounds exactly as the FP64 detection forms them
                    auto blo_at = [&](int v) {
                        const double lo = bnd[2 * v], hi = bnd[2 * v + 1];
                        return lo - fmax(1e-4, 1e-3 * (hi - lo));
                    };
                    auto bhi_at = [&](int v) {
                        const double lo = bnd[2 * v], hi = bnd[2 * v + 1];
                        return hi + fmax(1e-4, 1e-3 * (hi - lo));
                    };
                    float dlo[L::M], ulo[L::M], dhi[L::M], uhi[L::M];
#pragma unroll
                    for (int v = 0; v < L::M; ++v) {
                        const float rlo = __shfl_sync(0xffffffffu, rlo_l, v), rhi = __shfl_sync(0xffffffffu, rhi_l, v);
                        const float tol = __shfl_sync(0xffffffffu, tol_l, v);
                        dlo[v] = rlo - tol;
                        ulo[v] = rlo + tol;
                        dhi[v] = rhi - tol;
                        uhi[v] = rhi + tol;
                    }
                    for (int a = lane; a < L::NSUB; a += 32) {
                        float x[L::M];
                        NodeIO<float, L::M>::load(avg + a * L::M, x);
                        int close = 0;
#pragma unroll
                        for (int v = 0; v < L::M; ++v) {
                            bad |= x[v] < dlo[v] || x[v] > uhi[v];
                            close |= (x[v] < ulo[v] || x[v] > dhi[v]) ? (1 << v) : 0;
                        }
                        if (close && !bad) {  // too close to call in FP32: FP64 averages
#pragma unroll 1
                            for (int v = 0; v < L::M; ++v) {
                                if (!((close >> v) & 1)) continue;
                                const double x64 = lim_average64<L, DIM>(uc, Pr64, a, v);
                                const double blo = blo_at(v), bhi = bhi_at(v);
                                bad |= x64 < blo || x64 > bhi;
                            }
                        }
                    }
                    bad = __any_sync(0xffffffffu, bad);
                }
                if (lane == 0) {
                    S.lim_flags[e] = bad;
                    if (bad) {
                        // at most E entries a step (the reset after the limiter empties it)
                        const unsigned k = atomicAdd(&S.ctl->lim_count, 1u);
                        if (k < (unsigned)S.E) {
                            S.lim_list[k] = (int)e;
                            if (S.lim_slot) S.lim_slot[e] = (int)k;
                        }
                    }
                }
                __syncwarp();
            }
        }
    }
}

template <class PDE, int DIM, int N>
__global__ void __launch_bounds__(128) k_lim_fv(const KParams P)
{
    using L = LimCfg<PDE, DIM, N>;
    if constexpr (L::OK) {
        constexpr int M = L::M, S_ = L::S;
        if (!lim_any_troubled(P)) return;  // uniform over the grid
        extern __shared__ __align__(16) unsigned char smem_raw[];
        LimSmem<L> sm(reinterpret_cast<double *>(smem_raw));
        lim_load_ops<L>(P, sm);
        for (int si = 0; si < P.nsolves; ++si) {
            const SolveDesc &S = P.solves[si];
            if (!S.u_prev) continue;
            const double dt = solve_dt(P, S);
            if (!(dt > 0.0)) continue;
            // the troubled elements, one per CTA (their order does not
            // matter: each is computed on its own)
            const unsigned ntroubled = min(S.ctl->lim_count, (unsigned)S.E);
            for (unsigned k = blockIdx.x; k < ntroubled; k += gridDim.x) {
                const long long e = S.lim_list[k];
                lim_un_averages<L, DIM>(S, e, sm, sm.avg);
#pragma unroll 1
                for (int d = 0; d < DIM; ++d)
#pragma unroll 1
                    for (int side = 0; side < 2; ++side) {
                        const long long nb = neighbour_of(S, (int)e, d, side ? 1 : -1);
                        lim_un_averages<L, DIM>(S, nb, sm, sm.nb);
                        // ghost cells -2, -1 from the lower neighbour's last
                        // layers; S, S+1 from the upper neighbour's first ones
                        lim_layers<L, DIM>(sm.nb, d, side ? 0 : 1,
                                           sm.ghost + (size_t)(d * 2 + side) * 2 * L::NLINE * M);
                        __syncthreads();
                    }
                // sm.nb is free from here on: the source's sum over directions of
                // the half-step changes
                double *ctr = sm.nb;
                for (int i = threadIdx.x; i < L::NSUB * M; i += blockDim.x) sm.dq[i] = ctr[i] = 0.0;
                __syncthreads();
                // one direction at a time, d a compile-time constant (the fluxes
                // of the other directions are then never formed)
                auto direction = [&](auto dc) {
                    constexpr int d = decltype(dc)::value;
                    const double r = dt * S.inv_dx[d] * S_;  // dt / subcell width
                    // cell i of line l along d: ghost layers below 0 and from S on
                    auto cell = [&](int l, int i) -> const double * {
                        if (i < 0) return sm.ghost + ((size_t)((d * 2 + 0) * 2 + (i + 2)) * L::NLINE + l) * M;
                        if (i >= S_) return sm.ghost + ((size_t)((d * 2 + 1) * 2 + (i - S_)) * L::NLINE + l) * M;
                        return sm.avg + lim_cell<DIM, S_>(d, l, i) * M;
                    };
                    // every face of this direction (face f between cells f-1 and f):
                    // the flux, or the two fluctuations [lower | upper]
                    constexpr int FW = PDE::NCP ? 2 * M : M;
                    // the element's own boundary faces (f = 0, S) are kept for the
                    // coupling of its unlimited neighbours when the solve has a slot
                    double *keep = S.lim_fb && (long long)k < S.lim_fb_slots
                                       ? S.lim_fb + (long long)k * L::FB_SLOT + (size_t)d * 2 * L::NLINE * L::FB
                                       : nullptr;
                    for (int it = threadIdx.x; it < (S_ + 1) * L::NLINE; it += blockDim.x) {
                        const int f = it % (S_ + 1), l = it / (S_ + 1);
                        double *fo = sm.fb + (size_t)it * FW;
                        // the record of a boundary face: [side][line][FB]
                        double *rec = keep && (f == 0 || f == S_) ? keep + ((size_t)(f ? 1 : 0) * L::NLINE + l) * L::FB
                                                                  : nullptr;
                        if constexpr (PDE::NCP) {
                            // the neighbour's own state at the face: the lower cell's
                            // evolved value at f = 0, the upper one's at f = S
                            lim_face_nc<PDE, DIM>(P.pde, cell(l, f - 2), cell(l, f - 1), cell(l, f), cell(l, f + 1),
                                                  d, r, dt, fo, fo + M, rec && f == 0 ? rec + M : nullptr,
                                                  rec && f == S_ ? rec + M : nullptr);
                            if (rec) {
#pragma unroll
                                for (int v = 0; v < M; ++v) rec[v] = f == 0 ? fo[v] : fo[M + v];
                            }
                        } else {
                            lim_face<PDE, DIM>(P.pde, cell(l, f - 2), cell(l, f - 1), cell(l, f), cell(l, f + 1), d, r,
                                               dt, fo);
                            if (rec) {
#pragma unroll
                                for (int v = 0; v < M; ++v) rec[v] = fo[v];
                            }
                        }
                    }
                    __syncthreads();
                    for (int it = threadIdx.x; it < S_ * L::NLINE; it += blockDim.x) {
                        const int i = it % S_, l = it / S_;
                        const double *F0 = sm.fb + (size_t)(l * (S_ + 1) + i) * FW, *F1 = F0 + FW;
                        const int k = lim_cell<DIM, S_>(d, l, i);
                        double *o = sm.dq + k * M;
                        if constexpr (PDE::NCP) {
                            // F1: the lower cell's fluctuation of face i+1; F0 + M:
                            // the upper cell's of face i; then the smooth part of
                            // B(q) grad q inside the subcell at its half-step centre
                            double sl[M], chc[M], cw[M], Bc[M];
                            const double *w = cell(l, i);
                            lim_half<PDE, DIM>(P.pde, cell(l, i - 1), w, cell(l, i + 1), d, r, dt, sl, nullptr, nullptr,
                                               chc);
#pragma unroll
                            for (int v = 0; v < M; ++v) cw[v] = w[v] + chc[v];
                            lim_bdot<PDE>(cw, d, sl, Bc);
#pragma unroll
                            for (int v = 0; v < M; ++v) {
                                o[v] -= r * (F1[v] - F0[M + v]);
                                o[v] -= r * Bc[v];
                            }
                        } else {
#pragma unroll
                            for (int v = 0; v < M; ++v) o[v] -= r * (F1[v] - F0[v]);
                        }
                        if constexpr (PDE::HAS_SRC) {
                            double chc[M];
                            lim_half<PDE, DIM>(P.pde, cell(l, i - 1), cell(l, i), cell(l, i + 1), d, r, dt, nullptr,
                                               nullptr, nullptr, chc);
#pragma unroll
                            for (int v = 0; v < M; ++v) ctr[k * M + v] += chc[v];
                        }
                    }
                    __syncthreads();
                };
                direction(std::integral_constant<int, 0>{});
                if constexpr (DIM > 1) direction(std::integral_constant<int, 1>{});
                if constexpr (DIM > 2) direction(std::integral_constant<int, 2>{});
                if constexpr (PDE::HAS_SRC) {
                    // the source at the half-step centre of all directions
                    for (int a = threadIdx.x; a < L::NSUB; a += blockDim.x) {
                        double S0[M], S1[M], w[M];
                        const double *av = sm.avg + a * M;
                        PDE::source(P.pde, av, S0);
#pragma unroll
                        for (int v = 0; v < M; ++v) w[v] = av[v] + ctr[a * M + v] + 0.5 * dt * S0[v];
                        PDE::source(P.pde, w, S1);
#pragma unroll
                        for (int v = 0; v < M; ++v) sm.dq[a * M + v] += dt * S1[v];
                    }
                    __syncthreads();
                }
                for (int i = threadIdx.x; i < L::NSUB * M; i += blockDim.x) sm.dq[i] += sm.avg[i];
                __syncthreads();
                if (S.lim_subn)  // kept: the next step's subcell data of e
                    for (int i = threadIdx.x; i < L::NSUB * M; i += blockDim.x)
                        S.lim_subn[e * (L::NSUB * M) + i] = sm.dq[i];
                lim_tensor<DIM, M, L::n, S_>(sm.dq, sm.u, sm.ta, sm.tb, sm.Rc);
                // the material fields (q_t = 0) are kept as they were
                for (int i = threadIdx.x; i < L::NS * M; i += blockDim.x)
                    S.u_out[e * (L::NS * M) + i] = (i % M) < PDE::MEV ? sm.u[i] : S.u_prev[e * (L::NS * M) + i];
                __syncthreads();
            }
        }
    }
}

// T: the compute type of the step whose face fluxes are replaced (double:
// FP64 trace records; float: the FP32 path's perturbation records about
// each element's reference state).
template <class PDE, int DIM, int N, typename T = double>
__global__ void __launch_bounds__(128) k_lim_couple(const KParams P)
{
    using L = LimCfg<PDE, DIM, N>;
    if constexpr (L::OK) {
        constexpr int M = L::M, S_ = L::S, n = L::n, NF = L::NF, RS = Geom<PDE, DIM, N>::RS;
        constexpr int NFACE = 2 * DIM * NF;
        if (!lim_any_troubled(P)) return;  // uniform over the grid
        extern __shared__ __align__(16) unsigned char smem_raw[];
        LimSmem<L> sm(reinterpret_cast<double *>(smem_raw));
        lim_load_ops<L>(P, sm);
        for (int si = 0; si < P.nsolves; ++si) {
            const SolveDesc &S = P.solves[si];
            if (!S.u_prev) continue;
            const double dt = solve_dt(P, S);
            if (!(dt > 0.0)) continue;
            if (S.ctl->lim_count == 0u) continue;  // no troubled element this step: nothing to couple
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                // the limited state's wave-speed maxima and non-finite flag
                // are taken afresh by k_cfl after this launch (nothing else
                // touches them meanwhile)
                for (int d = 0; d < 3; ++d) S.ctl->lam_acc[d] = 0ull;
                S.ctl->flags &= ~FLAG_NONFINITE;
            }
            const double *tr = reinterpret_cast<const double *>(S.tr);
            for (long long e = blockIdx.x; e < S.E; e += gridDim.x) {
                if (S.lim_flags[e]) continue;
                int any = 0;
#pragma unroll
                for (int d = 0; d < DIM; ++d)
#pragma unroll
                    for (int side = 0; side < 2; ++side)
                        any |= S.lim_flags[neighbour_of(S, (int)e, d, side ? 1 : -1)];
                if (!any) continue;  // uniform over the CTA
                bool own = false;  // this element's subcell averages in sm.avg
#pragma unroll 1
                for (int d = 0; d < DIM; ++d)
#pragma unroll 1
                    for (int side = 0; side < 2; ++side) {
                        const long long nb = neighbour_of(S, (int)e, d, side ? 1 : -1);
                        if (!S.lim_flags[nb]) continue;
                        // the troubled neighbour's subcell fluxes on this face as its
                        // subcell scheme formed them (its face toward this element:
                        // side 0 when this element is below it), or, beyond the
                        // solve's slots, formed here from the same subcell averages
                        // with the same function
                        const long long slot = S.lim_fb ? (long long)S.lim_slot[nb] : S.lim_fb_slots;
                        const double *stored =
                            slot < S.lim_fb_slots
                                ? S.lim_fb + slot * (long long)L::FB_SLOT + ((size_t)d * 2 + (side ? 0 : 1)) * L::NLINE * L::FB
                                : nullptr;  // uniform over the CTA
                        // the face's four cell layers: lower element's last two,
                        // upper element's first two
                        double *gl = sm.ghost, *gu = sm.ghost + 2 * L::NLINE * M;
                        if (!stored) {
                            if (!own) {
                                lim_un_averages<L, DIM>(S, e, sm, sm.avg);
                                own = true;
                            }
                            lim_un_averages<L, DIM>(S, nb, sm, sm.nb);
                            lim_layers<L, DIM>(side ? sm.avg : sm.nb, d, 1, gl);
                            lim_layers<L, DIM>(side ? sm.nb : sm.avg, d, 0, gu);
                            __syncthreads();
                        }
                        const double r = dt * S.inv_dx[d] * S_;
                        const long long el = side ? e : nb, eu = side ? nb : e;
                        // per face node: projected subcell flux minus the DG flux
                        if constexpr (PDE::NCP) {
                            // per line: the fluctuation this element receives and
                            // its own subcell state at the face [line][2M]
                            double *Fl = sm.dq, *dF = sm.dq + (size_t)L::NLINE * 2 * M;  // dF: [p][v]
                            for (int l = threadIdx.x; l < L::NLINE; l += blockDim.x) {
                                double *o = Fl + (size_t)l * 2 * M;
                                if (stored) {
#pragma unroll
                                    for (int v = 0; v < 2 * M; ++v) o[v] = stored[(size_t)l * 2 * M + v];
                                    continue;
                                }
                                const double *a0 = gl + (size_t)l * M, *a1 = gl + (size_t)(L::NLINE + l) * M;
                                const double *b0 = gu + (size_t)l * M, *b1 = gu + (size_t)(L::NLINE + l) * M;
                                if (side)  // this element is the lower one
                                    lim_face_nc<PDE, DIM>(P.pde, a0, a1, b0, b1, d, r, dt, o, nullptr, o + M, nullptr);
                                else
                                    lim_face_nc<PDE, DIM>(P.pde, a0, a1, b0, b1, d, r, dt, nullptr, o, nullptr, o + M);
                            }
                            __syncthreads();
                            // per (face node, line): the projected fluctuation plus
                            // the path integral from this element's DG trace to its
                            // subcell state at the face, into sm.fb [p][line][v]
                            static_assert((size_t)NF * L::NLINE * M <= (size_t)L::FACES, "coupling terms exceed sm.fb");
                            double *Cp = sm.fb;
                            for (int it = threadIdx.x; it < NF * L::NLINE; it += blockDim.x) {
                                const int l = it % L::NLINE, p = it / L::NLINE;
                                int pk[3], rem = p;
#pragma unroll
                                for (int k = 0; k < DIM - 1; ++k) {
                                    pk[k] = rem % n;
                                    rem /= n;
                                }
                                double wgt = 1.0;
                                int lr = l;
#pragma unroll
                                for (int k = 0; k < DIM - 1; ++k) {
                                    const int j = lr % S_;
                                    lr /= S_;
                                    wgt *= sm.Pr[j * n + pk[k]] / S_ / P.b.w[pk[k]];
                                }
                                const long long orec = side ? (el * NFACE + (d * 2 + 1) * NF + p) * RS
                                                            : (eu * NFACE + (d * 2 + 0) * NF + p) * RS;
                                double qown[M];  // this element's DG trace
                                if constexpr (sizeof(T) == 4) {  // perturbation about its reference
                                    const T *qd = reinterpret_cast<const T *>(S.tr) + orec;
#pragma unroll
                                    for (int v = 0; v < M; ++v) qown[v] = widen<T>(qd[v]) + S.ref[e * M + v];
                                } else {
#pragma unroll
                                    for (int v = 0; v < M; ++v) qown[v] = tr[orec + v];
                                }
                                const double *fs = Fl + (size_t)l * 2 * M;
                                double dq[M], J[M];
#pragma unroll
                                for (int v = 0; v < M; ++v) dq[v] = fs[M + v] - qown[v];
                                PDE::path_jump(qown, dq, d, J);
#pragma unroll
                                for (int v = 0; v < M; ++v) Cp[(size_t)it * M + v] = wgt * (fs[v] + J[v]);
                            }
                            __syncthreads();
                            for (int p = threadIdx.x; p < NF; p += blockDim.x) {
                                double Ft[M], dq[M], J[M];
#pragma unroll
                                for (int v = 0; v < M; ++v) Ft[v] = 0.0;
                                for (int l = 0; l < L::NLINE; ++l)
#pragma unroll
                                    for (int v = 0; v < M; ++v) Ft[v] += Cp[((size_t)p * L::NLINE + l) * M + v];
                                // the corrector's path-conservative fluctuation on this face node
                                if constexpr (sizeof(T) == 4) {
                                    // as the FP32 corrector forms it: perturbation records
                                    // about each element's reference, the lower state and
                                    // the jump made absolute with the reference difference
                                    const T *trf = reinterpret_cast<const T *>(S.tr);
                                    const T *Lq = trf + (el * NFACE + (d * 2 + 1) * NF + p) * RS;
                                    const T *Rq = trf + (eu * NFACE + (d * 2 + 0) * NF + p) * RS;
                                    const T smax = tmax(Lq[Geom<PDE, DIM, N>::LAM], Rq[Geom<PDE, DIM, N>::LAM]);
                                    const double *ro = S.ref + e * M, *rn = S.ref + nb * M;
                                    const T sg = side ? T(1) : T(-1);
                                    T dqf[M], qa[M], Jf[M];
#pragma unroll
                                    for (int v = 0; v < M; ++v) {
                                        const T dlq = sg * narrow<T>(rn[v] - ro[v]);
                                        dqf[v] = Rq[v] - Lq[v];
                                        qa[v] = Lq[v];
                                        dqf[v] += dlq;
                                        qa[v] += narrow<T>(ro[v]) - (side ? T(0) : dlq);
                                    }
                                    PDE::path_jump(qa, dqf, d, Jf);
                                    const T hs = side ? T(0.5) : T(-0.5);
#pragma unroll
                                    for (int v = 0; v < M; ++v) {
                                        const T f = hs * Jf[v] - T(0.5) * smax * dqf[v];
                                        dF[p * M + v] = Ft[v] - (v < PDE::MEV ? widen<T>(f) : 0.0);
                                    }
                                } else {
                                    const double *Lr = tr + (el * NFACE + (d * 2 + 1) * NF + p) * RS;
                                    const double *Rr = tr + (eu * NFACE + (d * 2 + 0) * NF + p) * RS;
                                    const double smax = tmax(Lr[Geom<PDE, DIM, N>::LAM], Rr[Geom<PDE, DIM, N>::LAM]);
#pragma unroll
                                    for (int v = 0; v < M; ++v) dq[v] = Rr[v] - Lr[v];
                                    PDE::path_jump(Lr, dq, d, J);
                                    const double hs = side ? 0.5 : -0.5;
#pragma unroll
                                    for (int v = 0; v < M; ++v)
                                        dF[p * M + v] = Ft[v] - (v < PDE::MEV ? hs * J[v] - 0.5 * smax * dq[v] : 0.0);
                                }
                            }
                            __syncthreads();
                        } else if constexpr (sizeof(T) == 4) {
                            double *Fl = sm.dq;  // subcell fluxes on the face [line][v]
                            for (int l = threadIdx.x; l < L::NLINE; l += blockDim.x) {
                                if (stored) {
#pragma unroll
                                    for (int v = 0; v < M; ++v) Fl[(size_t)l * M + v] = stored[(size_t)l * M + v];
                                } else {
                                    lim_face<PDE, DIM>(P.pde, gl + (size_t)l * M, gl + (size_t)(L::NLINE + l) * M,
                                                       gu + (size_t)l * M, gu + (size_t)(L::NLINE + l) * M, d, r, dt,
                                                       Fl + (size_t)l * M);
                                }
                            }
                            __syncthreads();
                            double *dF = sm.dq + (size_t)L::NLINE * M;  // [p][v]
                            const T *trf = reinterpret_cast<const T *>(S.tr);
                            constexpr int LAM = Geom<PDE, DIM, N>::LAM;
                            for (int p = threadIdx.x; p < NF; p += blockDim.x) {
                                int pk[3], rem = p;
#pragma unroll
                                for (int k = 0; k < DIM - 1; ++k) {
                                    pk[k] = rem % n;
                                    rem /= n;
                                }
                                // the corrector's FP32 Rusanov flux of this element on this face
                                // node, formed as the corrector forms it: perturbation traces plus
                                // the reference differences across the face
                                const T *Lq = trf + (el * NFACE + (d * 2 + 1) * NF + p) * RS;
                                const T *Rq = trf + (eu * NFACE + (d * 2 + 0) * NF + p) * RS;
                                const T smax = tmax(Lq[LAM], Rq[LAM]);
                                const double *ro = S.ref + e * M, *rn = S.ref + nb * M;
                                T qf[M], dq[M], dFr[DIM][M];
#pragma unroll
                                for (int v = 0; v < M; ++v) {
                                    qf[v] = narrow<T>(ro[v]);
                                    dq[v] = narrow<T>(rn[v] - ro[v]);
                                }
                                typename PDE::template Ref<T> rr;
                                PDE::make_ref(P.pde, qf, rr);
                                PDE::flux_delta(P.pde, rr, dq, dFr);
                                // plus the element's reference flux, which the perturbation form
                                // leaves out of both its volume and its surface terms
                                double Fref[DIM][M];
                                PDE::flux(P.pde, ro, Fref);
                                const T sg = side ? T(1) : T(-1);
#pragma unroll
                                for (int v = 0; v < M; ++v) {
                                    T df = dFr[0][v];
                                    double fr = Fref[0][v];
#pragma unroll
                                    for (int k = 1; k < DIM; ++k) {
                                        df = d == k ? dFr[k][v] : df;
                                        fr = d == k ? Fref[k][v] : fr;
                                    }
                                    T f = T(0.5) * (Lq[M + v] + Rq[M + v]) - T(0.5) * smax * (Rq[v] - Lq[v]);
                                    f += (side ? T(0.5) : T(-0.5)) * (sg * df) - T(0.5) * smax * (sg * dq[v]);
                                    double Ft = 0.0;
                                    for (int l = 0; l < L::NLINE; ++l) {
                                        double wgt = 1.0;
                                        int lr = l;
#pragma unroll
                                        for (int k = 0; k < DIM - 1; ++k) {
                                            const int j = lr % S_;
                                            lr /= S_;
                                            wgt *= sm.Pr[j * n + pk[k]] / S_ / P.b.w[pk[k]];
                                        }
                                        Ft += wgt * Fl[(size_t)l * M + v];
                                    }
                                    dF[p * M + v] = Ft - (widen<T>(f) + fr);
                                }
                            }
                            __syncthreads();
                        } else {
                            double *Fl = sm.dq;  // subcell fluxes on the face [line][v]
                            for (int l = threadIdx.x; l < L::NLINE; l += blockDim.x) {
                                if (stored) {
#pragma unroll
                                    for (int v = 0; v < M; ++v) Fl[(size_t)l * M + v] = stored[(size_t)l * M + v];
                                } else {
                                    lim_face<PDE, DIM>(P.pde, gl + (size_t)l * M, gl + (size_t)(L::NLINE + l) * M,
                                                       gu + (size_t)l * M, gu + (size_t)(L::NLINE + l) * M, d, r, dt,
                                                       Fl + (size_t)l * M);
                                }
                            }
                            __syncthreads();
                            double *dF = sm.dq + (size_t)L::NLINE * M;  // [p][v]
                            for (int i = threadIdx.x; i < NF * M; i += blockDim.x) {
                                const int v = i % M, p = i / M;
                                int pk[3], rem = p;
#pragma unroll
                                for (int k = 0; k < DIM - 1; ++k) {
                                    pk[k] = rem % n;
                                    rem /= n;
                                }
                                double Ft = 0.0;
                                for (int l = 0; l < L::NLINE; ++l) {
                                    double wgt = 1.0;
                                    int lr = l;
#pragma unroll
                                    for (int k = 0; k < DIM - 1; ++k) {
                                        const int j = lr % S_;
                                        lr /= S_;
                                        wgt *= sm.Pr[j * n + pk[k]] / S_ / P.b.w[pk[k]];
                                    }
                                    Ft += wgt * Fl[(size_t)l * M + v];
                                }
                                // the corrector's Rusanov flux on this face node (lower | upper)
                                const double *Lr = tr + (el * NFACE + (d * 2 + 1) * NF + p) * RS;
                                const double *Rr = tr + (eu * NFACE + (d * 2 + 0) * NF + p) * RS;
                                const double smax = tmax(Lr[Geom<PDE, DIM, N>::LAM], Rr[Geom<PDE, DIM, N>::LAM]);
                                const double Fdg = 0.5 * (Lr[M + v] + Rr[M + v]) - 0.5 * smax * (Rr[v] - Lr[v]);
                                dF[i] = Ft - Fdg;
                            }
                            __syncthreads();
                        }
                        const double *dF = sm.dq + (size_t)L::NLINE * M * (PDE::NCP ? 2 : 1);
                        for (int i = threadIdx.x; i < L::NS * M; i += blockDim.x) {
                            const int v = i % M, s = i / M;
                            int sd = 0, p = 0, pw = 1, rem = s;
#pragma unroll
                            for (int k = 0; k < DIM; ++k) {
                                const int x = rem % n;
                                rem /= n;
                                if (k == d) {
                                    sd = x;
                                } else {
                                    p += x * pw;
                                    pw *= n;
                                }
                            }
                            const double lift = (side ? P.b.F1[sd] : -P.b.F0[sd]) * S.inv_dx[d] * P.b.inv_w[sd];
                            S.u_out[e * (L::NS * M) + i] -= dt * lift * dF[p * M + v];
                        }
                        __syncthreads();
                    }
            }
        }
    }
}

// Kept subcell data: a state given as the subcell averages of every element
// (uploaded to lim_subn).  Each element's nodal state becomes their
// least-squares reconstruction (R28) and every element is marked as limited,
// so that the next step takes the averages as its subcell data at t^n and
// the wave speeds of the state (k_cfl) come from them.  One solve, one
// element per CTA.
template <class PDE, int DIM, int N>
__global__ void __launch_bounds__(128) k_lim_subcell_init(const KParams P)
{
    using L = LimCfg<PDE, DIM, N>;
    if constexpr (L::OK) {
        constexpr int M = L::M;
        extern __shared__ __align__(16) unsigned char smem_raw[];
        LimSmem<L> sm(reinterpret_cast<double *>(smem_raw));
        lim_load_ops<L>(P, sm);
        const SolveDesc &S = P.solves[0];
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            S.ctl->lim_count = (unsigned)S.E;
            S.ctl->lim_kept_ok = 1u;
            S.ctl->lim_fresh = 0u;
        }
        for (long long e = blockIdx.x; e < S.E; e += gridDim.x) {
            const double *src = S.lim_subn + e * (L::NSUB * M);
            for (int i = threadIdx.x; i < L::NSUB * M; i += blockDim.x) sm.dq[i] = src[i];
            __syncthreads();
            lim_tensor<DIM, M, L::n, L::S>(sm.dq, sm.u, sm.ta, sm.tb, sm.Rc);
            for (int i = threadIdx.x; i < L::NS * M; i += blockDim.x) S.u_out[e * (L::NS * M) + i] = sm.u[i];
            if (threadIdx.x == 0) {
                S.lim_flags[e] = 1;
                S.lim_list[e] = (int)e;
            }
            __syncthreads();
        }
    }
}
