// Element-batch kernels of the ADER-DG step, templated on the PDE, the
// dimension, the degree and the compute type T (double: FP64 path; float:
// mixed path whose state update stays in double).
//
//  k_predictor  space-time predictor (Sec. 2.2, eq. pde.st2) by Picard
//               iteration, time averages, volume integral, face traces
//  k_corrector  Rusanov fluxes on the time-averaged traces (eq. pc.scheme
//               with B = 0, eq. rusanov), surface lift and element update
//               (eq. pde.nc.gw2), wave-speed maxima for the next CFL step
//  k_cfl        wave-speed maxima of a state (first step after an upload)
//
// Every launch serves a list of independent solves (same PDE, dimension
// and degree; any mesh size and spacing) described by SolveDesc entries in
// device memory.  The launch's tiles -- EPB consecutive elements of one
// solve -- are numbered solve after solve; a CTA finds its solve by binary
// search over the tile offsets and loops over tiles with a grid stride, so
// the grid can be sized to the GPU (persistent) or to the tile count.
// Within a tile the element working set stays in shared memory and
// registers: u^n is read once and the space-time DOFs never reach HBM (the
// cache-blocking property of Sec. 2.2 mapped onto an SM).
#pragma once

#include "common.cuh"

namespace aderdg {

template <typename T>
__device__ __forceinline__ T tmax(T a, T b) { return a > b ? a : b; }

__host__ __device__ constexpr int cmin(int a, int b) { return a < b ? a : b; }
__host__ __device__ constexpr int cmax(int a, int b) { return a > b ? a : b; }
__host__ __device__ constexpr int cgcd(int a, int b) { return b == 0 ? a : cgcd(b, a % b); }
__host__ __device__ constexpr size_t align16(size_t b) { return (b + 15) / 16 * 16; }

// Load/store the M values of one node with the widest vector access the
// node size allows (float4 for 4 floats, 2 x double2 for 4 doubles, ...).
template <int B> struct VecOf;
template <> struct VecOf<16> { using t = float4; };
template <> struct VecOf<8> { using t = float2; };
template <> struct VecOf<4> { using t = float; };

template <typename T, int M>
struct NodeIO {
    static constexpr int BYTES = (int)sizeof(T) * M;
    static constexpr int VB = BYTES % 16 == 0 ? 16 : (BYTES % 8 == 0 ? 8 : (int)sizeof(T));
    static constexpr int K = VB / (int)sizeof(T);  // values per access
    using VT = typename VecOf<VB>::t;
    __device__ __forceinline__ static void load(const T *p, T *x)
    {
#pragma unroll
        for (int i = 0; i < M / K; ++i) {
            const VT w = reinterpret_cast<const VT *>(p)[i];
            const T *ws = reinterpret_cast<const T *>(&w);
#pragma unroll
            for (int k = 0; k < K; ++k) x[i * K + k] = ws[k];
        }
    }
    __device__ __forceinline__ static void store(T *p, const T *x)
    {
#pragma unroll
        for (int i = 0; i < M / K; ++i) {
            VT w;
            T *ws = reinterpret_cast<T *>(&w);
#pragma unroll
            for (int k = 0; k < K; ++k) ws[k] = x[i * K + k];
            reinterpret_cast<VT *>(p)[i] = w;
        }
    }
};

// Tile -> solve: the last solve whose first tile is <= tile.
__device__ __forceinline__ int find_solve(const SolveDesc *S, int nsolves, long long tile, int which)
{
    int lo = 0, hi = nsolves - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        const long long t0 = which ? S[mid].tile0_c : S[mid].tile0_p;
        if (t0 <= tile) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ double solve_dt(const KParams &P, const SolveDesc &S)
{
    return P.use_ctl_dt ? S.ctl->dt : P.dt_arg;
}

// Non-finite test and float <-> double conversions on the integer bits, so
// that the FP64 pipe only carries the arithmetic the method needs in FP64.
__device__ __forceinline__ bool dbl_nonfinite(double x)
{
    return ((__double2hiint(x) >> 20) & 0x7ff) == 0x7ff;
}

// double -> float, round to nearest even (an unbiased rounding: the FP32
// path accumulates these values over many steps); results below the normal
// float range become signed zero, beyond it signed infinity
__device__ __forceinline__ float dbl_to_flt_rn(double x)
{
    const int hi = __double2hiint(x);
    const unsigned lo = (unsigned)__double2loint(x);
    const unsigned sign = (unsigned)hi & 0x80000000u;
    const int e = ((hi >> 20) & 0x7ff) - 1023 + 127;
    const unsigned mant = (((unsigned)hi & 0xfffffu) << 3) | (lo >> 29);
    const unsigned rem = lo & 0x1fffffffu;
    unsigned bits = ((unsigned)e << 23) | mant;
    bits += (rem > 0x10000000u || (rem == 0x10000000u && (mant & 1u))) ? 1u : 0u;  // may carry into e
    bits |= sign;
    bits = e <= 0 ? sign : bits;
    bits = (e >= 255 || (bits & 0x7f800000u) == 0x7f800000u) ? (sign | 0x7f800000u) : bits;
    return __uint_as_float(bits);
}

// float -> double widening on the integer bits (exact for normal numbers and
// zero; FP32 denormals, which the FP32 path never produces at these
// magnitudes, are flushed to zero)
__device__ __forceinline__ double flt_to_dbl(float f)
{
    const unsigned b = __float_as_uint(f);
    const unsigned e = (b >> 23) & 0xffu;
    const unsigned long long sign = (unsigned long long)(b & 0x80000000u) << 32;
    unsigned long long bits = sign | ((unsigned long long)(e + 896u) << 52) |
                              ((unsigned long long)(b & 0x7fffffu) << 29);
    bits = e == 0 ? sign : bits;
    bits = e == 0xffu ? (sign | 0x7ff0000000000000ull | ((unsigned long long)(b & 0x7fffffu) << 29)) : bits;
    return __longlong_as_double((long long)bits);
}

template <typename T>
__device__ __forceinline__ double widen(T x);
template <>
__device__ __forceinline__ double widen<double>(double x) { return x; }
template <>
__device__ __forceinline__ double widen<float>(float x) { return flt_to_dbl(x); }

template <typename T>
__device__ __forceinline__ T narrow(double x);
template <>
__device__ __forceinline__ double narrow<double>(double x) { return x; }
template <>
__device__ __forceinline__ float narrow<float>(double x) { return dbl_to_flt_rn(x); }

// ===========================================================================
// Predictor
// ===========================================================================
//
// Thread (element g, spatial node s) owns the time pencil q[0..n)[0..M) of
// node s in registers.  One Picard iteration:
//   1. F_d(q[t]) at its n nodes -> shared buffer F_d[t][s][v]
//   2. each thread takes one d-pencil per direction (there are exactly NS of
//      them: n time levels x NF face positions) and overwrites it in place
//      with -Dhat F_d (the n x n operator is read from the parameter bank
//      with compile-time indices)
//   3. back on the time pencil: R = sum_d (1/dx_d) (-Dhat F_d),
//      q[t] = u + dt sum_t' iK1W[t][t'] R[t']
// Initial guesses (Sec. 2.2) need the flux of time-constant states only: one
// flux per spatial node and the t = 0 pencils.  From the trivial guess
// q = u the first iteration is taken that way, q[t] = u + dt c1[t] R with c1
// the row sums of iK1W (the general iteration applied to a time-constant
// q); the second- and third-order guesses are Taylor polynomials in
// tau = xi dt built from R(u) and R(u + dt L(u)).
template <class PDE, int DIM, int N, typename T, int TS = 0>
struct PredCfg {
    using G = Geom<PDE, DIM, N>;
    static constexpr int n = G::n, M = G::M, NS = G::NS, NST = G::NST, NF = G::NF, NREC = G::NREC;
    static constexpr int LAM = G::LAM;
    static constexpr int DIMS = DIM;
    // values per node in the exchange fields: all m (the flux F_d), or for a
    // purely non-conservative system its evolved variables (the material
    // fields enter B as coefficients; alpha's gradient, constant in time, is
    // taken once per tile)
    static constexpr int MX = PDE::NCP ? PDE::MEV : M;
    // variables whose time derivative can be nonzero (the rest keep q = u)
    static constexpr int MR = PDE::NCP ? PDE::MEV : M;
    // per-element shared buffer: DIM space-time flux fields, later
    // qbar | Fbar_d (| face states, where records outnumber threads)
    // Exchange field F_d[t][s][v] of an element: time slices TSL values apart
    // (NS m plus TPAD), directions FSL = n TSL apart.  3D FP32 with n = 4
    // pads every slice by one word and maps x-pencils t-fastest: a count of
    // the conflicting 4-byte bank accesses of the store / contract / gather
    // phases gives 7488 -> 4608 wavefronts per iteration and CTA for m = 9,
    // 4160 -> 3200 for m = 5, 832 -> 640 for m = 1 (no gain for other n).
    static constexpr bool PAD3 = (DIM == 3 && sizeof(T) == 4 && n == 4 && MX % 2 == 1);  // keeps scalar nodes
    static constexpr int TPAD = PAD3 ? 1 : 0;
    static constexpr int TSL = NS * MX + TPAD;
    static constexpr int FSL = n * TSL;
    // shapes 7 and 8 (FP32, conservative systems): the state q goes through
    // shared memory once (one more field) and each d-pencil owner takes F_d
    // of its own pencil, instead of every flux field going through it
    static constexpr bool QX = TS >= 7 && sizeof(T) == 4 && !PDE::NCP;
    static constexpr int ELEM0x =
        cmax((DIM + (QX ? 1 : 0)) * FSL + (PAD3 ? 1 : 0), ((1 + DIM) * NS + (NREC > NS ? NREC : 0)) * M);
    // the non-conservative layout's vector nodes (MX even) want every
    // element buffer 16-byte aligned
    static constexpr int ELEM0 = PDE::NCP ? round_up(ELEM0x, 4) : ELEM0x;
    // Shared-memory bank layout of the 2D FP32 path with 16-byte nodes
    // (Euler, m = 4), chosen per n from a bank-conflict count of the
    // store / contract / gather phases: bit 0 pads the per-element buffer to
    // 1 node mod 8 (neighbouring elements start on other banks), bit 1 maps
    // thread s to the x-pencil (t = s mod n, p = s / n) instead of
    // (t = s / n, p = s mod n).  Counted wavefronts per iteration and CTA,
    // before -> after: n = 3: 732 -> 576, n = 5: 920 -> 780, n = 6: 1044 ->
    // 1020, n = 7: 980 -> 952; n = 2, 4, 8 unchanged.
    static constexpr int BANKS = (DIM == 2 && sizeof(T) == 4 && M == 4)
                                     ? (n == 3 || n == 5 || n == 7 ? 3 : (n == 6 ? 1 : 0))
                                     : 0;
    static constexpr int ELEM = (BANKS & 1) ? ELEM0 + (((1 - ELEM0 / M) % 8 + 8) % 8) * M : ELEM0;
    static constexpr bool MAPB0 = (BANKS & 2) != 0 || PAD3;
    // Shape 0 -- FP64: smaller CTAs, several per SM (independent barrier
    // domains keep the DFMA pipe fed); FP32: 256-thread CTAs.  Shapes 1 and
    // 2 halve and double the CTA at the same register cap per thread.
    static constexpr int TARGET0 = sizeof(T) == 8 ? 128 : 256;
    static constexpr int MINB0 = PDE::NCP ? (sizeof(T) == 8 ? 1 : 2)
                                 : sizeof(T) == 8 ? (n * M < 24 ? 3 : 2) : ((n * M <= 20 || (M == 9 && n <= 4)) ? 3 : 2);
    // shapes 5 and 6: the CTA geometry of shapes 0 and 1 with the derivative
    // contractions on the tensor cores (FP32 path only; see contract_all_mma)
    static constexpr int TSG = TS >= 7 ? TS - 7 : (TS >= 5 ? TS - 5 : TS);
    static constexpr bool TC = TS >= 5 && TS <= 6 && sizeof(T) == 4 && n <= 8;
    static constexpr int TARGET = TSG == 1 ? TARGET0 / 2 : (TSG == 2 ? TARGET0 * 2 : TARGET0);
    static constexpr int EPB_S = cmax(1, (int)((110 * 1024) / (ELEM * sizeof(T))));
    static constexpr int EPB = cmin(cmax(1, TARGET / NS), EPB_S);
    static constexpr int THREADS = round_up(EPB * NS, 32);
    static constexpr int THREADS0 = round_up(cmin(cmax(1, TARGET0 / NS), EPB_S) * NS, 32);
    // resident CTAs per SM for the launch bounds: the register cap per
    // thread of shape 0 (65536 / (THREADS0 MINB0)) is kept
    static constexpr int MINB = cmax(1, cmin(2048 / THREADS, (THREADS0 * MINB0) / THREADS));
    static constexpr int SHARED = round_up(DIM * n * n + 2 * n + 1 + 2 * n * n, 4);  // Kw, F0, F1, dt/dx, W, iK1W dt/dx
    // every vector access of a node in the exchange fields and in qbar |
    // Fbar starts on its vector width
    static_assert((SHARED * sizeof(T)) % 16 == 0, "shared header alignment");
    static_assert((ELEM * sizeof(T)) % NodeIO<T, MX>::VB == 0 && (TSL * sizeof(T)) % NodeIO<T, MX>::VB == 0 &&
                      (FSL * sizeof(T)) % NodeIO<T, MX>::VB == 0,
                  "exchange-field alignment");
    static_assert((ELEM * sizeof(T)) % NodeIO<T, M>::VB == 0, "element buffer alignment");
    static constexpr size_t BYTES = sizeof(T) * (size_t)(SHARED + EPB * ELEM);
    // FP32 path: perturbation form about the element's node SREF
    static constexpr bool DELTA = sizeof(T) == 4;
    static constexpr int SREF = NS / 2;
    static constexpr int RF = M;  // reference record: q_ref
};

// Weights of the extrapolation guess: W[t][k] = L_k(1 + xi_t r) - L_k(1),
// L_k the Lagrange basis of the time nodes (barycentric weights bw), r =
// dt / dt_prev.  One thread; compile-time indices into the operator table.
template <typename T, int n>
__device__ __forceinline__ void extrap_weights(const Ops<T> &O, T r, T *W)
{
#pragma unroll
    for (int t = 0; t < n; ++t) {
        const T x = T(1) + O.xi[t] * r;
#pragma unroll
        for (int k = 0; k < n; ++k) {
            T L = O.bw[k];
#pragma unroll
            for (int j = 0; j < n; ++j)
                if (j != k) L *= x - O.xi[j];
            W[t * n + k] = L - O.F1[k];
        }
    }
}

// -Dhat F_d along direction D on pencil (t, p), in place.
template <class C, int D, typename T>
__device__ __forceinline__ void contract_pencil(T *Fd, int t, int p, const T *Dm)
{
    constexpr int n = C::n, M = C::MX;
    constexpr int pd = ipow(n, D);
    using IO = NodeIO<T, M>;
    const int s0 = (p % pd) + (p / pd) * pd * n;
    T *base = Fd + t * C::TSL + s0 * M;
    T x[n][M];
#pragma unroll
    for (int j = 0; j < n; ++j) IO::load(base + j * pd * M, x[j]);
#pragma unroll
    for (int i = 0; i < n; ++i) {
        T y[M];
#pragma unroll
        for (int v = 0; v < M; ++v) {
            T acc = Dm[i * n] * x[0][v];
#pragma unroll
            for (int j = 1; j < n; ++j) acc += Dm[i * n + j] * x[j][v];
            y[v] = acc;
        }
        IO::store(base + i * pd * M, y);
    }
}

// Every direction's pencil (t, p) in place; direction 0 takes (t0, p0).
template <class C, typename T, int D = 0>
__device__ __forceinline__ void contract_all(T *ebuf, int t0, int p0, int t, int p, const Ops<T> &O)
{
    if constexpr (D < C::DIMS) {
        if constexpr (D == 0) contract_pencil<C, D, T>(ebuf, t0, p0, O.Dm[D]);
        else contract_pencil<C, D, T>(ebuf + D * C::FSL, t, p, O.Dm[D]);
        contract_all<C, T, D + 1>(ebuf, t0, p0, t, p, O);
    }
}

// -Dhat F_d along direction D on pencil (t, p) from the state field: the
// pencil's n nodes of q (field DIM), the flux F_D at each (the flux functor
// gives every direction; the others are dead code once it is inlined), the
// contraction, and the result into field D -- the same values as
// contract_pencil on the flux field.
template <class C, int D, typename T, class Flux>
__device__ __forceinline__ void contract_pencil_qx(T *ebuf, int t, int p, const T *Dm, Flux &flx)
{
    constexpr int n = C::n, M = C::M;
    constexpr int pd = ipow(n, D);
    const int s0 = (p % pd) + (p / pd) * pd * n;
    const T *qb = ebuf + C::DIMS * C::FSL + t * C::TSL + s0 * M;
    T f[n][M];
#pragma unroll
    for (int j = 0; j < n; ++j) {
        T x[M], F[C::DIMS][M];
        NodeIO<T, M>::load(qb + j * pd * M, x);
        flx(x, F);
#pragma unroll
        for (int v = 0; v < M; ++v) f[j][v] = F[D][v];
    }
    T *base = ebuf + D * C::FSL + t * C::TSL + s0 * M;
#pragma unroll
    for (int i = 0; i < n; ++i) {
        T y[M];
#pragma unroll
        for (int v = 0; v < M; ++v) {
            T acc = Dm[i * n] * f[0][v];
#pragma unroll
            for (int j = 1; j < n; ++j) acc += Dm[i * n + j] * f[j][v];
            y[v] = acc;
        }
        NodeIO<T, M>::store(base + i * pd * M, y);
    }
}

template <class C, typename T, class Flux, int D = 0>
__device__ __forceinline__ void contract_all_qx(T *ebuf, int t0, int p0, int t, int p, const Ops<T> &O, Flux &flx)
{
    if constexpr (D < C::DIMS) {
        if constexpr (D == 0) contract_pencil_qx<C, D, T>(ebuf, t0, p0, O.Dm[D], flx);
        else contract_pencil_qx<C, D, T>(ebuf, t, p, O.Dm[D], flx);
        contract_all_qx<C, T, Flux, D + 1>(ebuf, t0, p0, t, p, O, flx);
    }
}

// ---------------------------------------------------------------------------
// Derivative contractions on the tensor cores (FP32 path).  For direction
// d the exchange field holds, per element, NS MX "rows" (time level t,
// pencil p across d, variable v), each a pencil of n values along d.  A
// warp takes 16 rows as the A operand of mma.m16n8k8 (TF32, FP32
// accumulate), with the pencil index as K, and -Dhat (transposed) as the B
// operand, so D[row][i] = sum_j -Dhat[i][j] x_row[j].  K position k holds
// pencil node tau(k) = 2k (k < 4) or 2(k - 4) + 1 (k >= 4): a lane then
// loads nodes 2c and 2c + 1 of its two rows (c = lane mod 4) and receives
// the outputs at the same two nodes of the same rows, so the result goes
// back in place with no exchange between lanes.  FP32 accuracy comes from
// three TF32 products, x_hi B_hi + x_hi B_lo + x_lo B_hi, with x = x_hi +
// x_lo split by masking (B split once, by round-to-nearest conversions).
// ---------------------------------------------------------------------------
#ifdef __CUDACC__
__device__ __forceinline__ unsigned to_tf32(float x)
{
    unsigned r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1)
{
    asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};\n"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
#endif

// This lane's B fragment of -Dhat: b0 = B[k = c][i] = -Dhat[i][2c],
// b1 = B[k = c + 4][i] = -Dhat[i][2c + 1], i = lane / 4 (zero outside
// n x n), split into TF32 hi and lo parts.  Compile-time indices into the
// operator table, selected by lane.
struct TcOp {
    unsigned h0, h1, l0, l1;
};

template <int n>
__device__ __forceinline__ TcOp tc_operator(const float *Dm)
{
    const int lane = threadIdx.x & 31, i = lane >> 2, j = 2 * (lane & 3);
    float b0 = 0.f, b1 = 0.f;
#pragma unroll
    for (int ii = 0; ii < n; ++ii)
#pragma unroll
        for (int jj = 0; jj < n; ++jj) {
            b0 = (ii == i && jj == j) ? Dm[ii * n + jj] : b0;
            b1 = (ii == i && jj == j + 1) ? Dm[ii * n + jj] : b1;
        }
    TcOp o;
    o.h0 = to_tf32(b0);
    o.h1 = to_tf32(b1);
    o.l0 = to_tf32(b0 - __uint_as_float(o.h0));
    o.l1 = to_tf32(b1 - __uint_as_float(o.h1));
    return o;
}

// Every direction's contraction of every element of the CTA, in place
// (all threads of the CTA take part, warp by warp; elements start at
// sbase, ELEM values apart).
template <class C>
__device__ __forceinline__ void contract_all_mma(float *sbase, const TcOp &op)
{
    constexpr int n = C::n, MX = C::MX, NS = C::NS, NP = NS / n;
    constexpr int ROWS = NS * MX;  // rows per element and direction
    constexpr int R = C::EPB * ROWS;
    constexpr int TILES = (R + 15) / 16;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int j0 = 2 * (lane & 3);
#pragma unroll 1
    for (int item = warp; item < C::DIMS * TILES; item += nw) {
        const int d = item / TILES, tile = item - d * TILES;
        const int pd = d == 0 ? 1 : (d == 1 ? n : n * n);
        const int js = pd * MX;  // stride of a pencil's nodes
        float *rp[2];
        bool ok[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int r = tile * 16 + (lane >> 2) + 8 * h;
            ok[h] = r < R;
            const int rr = ok[h] ? r : 0;
            const int g = rr / ROWS, rem = rr - g * ROWS;
            const int v = rem % MX, q = rem / MX;
            const int p = q % NP, t = q / NP;
            const int s0 = (p % pd) + (p / pd) * pd * n;
            rp[h] = sbase + g * C::ELEM + d * C::FSL + t * C::TSL + s0 * MX + v;
        }
        // A fragment: a0 (row 0, node j0), a1 (row 1, j0), a2 (row 0, j0+1), a3 (row 1, j0+1)
        const bool in0 = j0 < n, in1 = j0 + 1 < n;
        float x[4];
        x[0] = (ok[0] && in0) ? rp[0][j0 * js] : 0.f;
        x[1] = (ok[1] && in0) ? rp[1][j0 * js] : 0.f;
        x[2] = (ok[0] && in1) ? rp[0][(j0 + 1) * js] : 0.f;
        x[3] = (ok[1] && in1) ? rp[1][(j0 + 1) * js] : 0.f;
        // split on the integer pipe: hi keeps the TF32 bits of x (x - hi is
        // then exact in FP32), lo goes in as it is (the MMA reads its TF32 bits)
        unsigned hi[4], lo[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            hi[k] = __float_as_uint(x[k]) & 0xffffe000u;
            lo[k] = __float_as_uint(x[k] - __uint_as_float(hi[k]));
        }
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        mma_tf32(acc, lo, op.h0, op.h1);  // small terms first
        mma_tf32(acc, hi, op.l0, op.l1);
        mma_tf32(acc, hi, op.h0, op.h1);
        // D fragment: c0 (row 0, node j0), c1 (row 0, j0+1), c2 (row 1, j0), c3 (row 1, j0+1)
        if (ok[0] && in0) rp[0][j0 * js] = acc[0];
        if (ok[0] && in1) rp[0][(j0 + 1) * js] = acc[1];
        if (ok[1] && in0) rp[1][j0 * js] = acc[2];
        if (ok[1] && in1) rp[1][(j0 + 1) * js] = acc[3];
    }
}

// -Dhat F_d on one variable v of the t = 0 pencil p along d, in place; item
// = (d, p, v) with v fastest, so that the DIM NF M items of an element
// spread over all its threads (the time-constant L evaluations of the
// initial guesses touch t = 0 only).  The operator is the same for every
// d (Ops::Dm[0]); the FMA order is contract_pencil's.
template <class C, typename T>
__device__ __forceinline__ void contract_item_t0(T *ebuf, int item, const T *Dm)
{
    constexpr int n = C::n, M = C::MX, NF = C::NF;
    const int d = item / (NF * M);
    const int r = item - d * (NF * M);
    const int p = r / M, v = r - p * M;
    const int pd = d == 0 ? 1 : (d == 1 ? n : n * n);
    const int s0 = (p % pd) + (p / pd) * pd * n;
    T *base = ebuf + d * C::FSL + s0 * M + v;
    T x[n];
#pragma unroll
    for (int j = 0; j < n; ++j) x[j] = base[j * pd * M];
#pragma unroll
    for (int i = 0; i < n; ++i) {
        T acc = Dm[i * n] * x[0];
#pragma unroll
        for (int j = 1; j < n; ++j) acc += Dm[i * n + j] * x[j];
        base[i * pd * M] = acc;
    }
}

// dx_0 R at time level t of node s: R_0 + sum_{d>0} (dx_0/dx_d) R_d (the
// factor 1/dx_0 is folded into dt by the caller, so isotropic and
// anisotropic meshes cost the same).
template <class C, typename T>
__device__ __forceinline__ void gather_R(const T *ebuf, int t, int s, const T *ratio, T *R)
{
    constexpr int M = C::M;
    NodeIO<T, M>::load(ebuf + t * C::TSL + s * M, R);
#pragma unroll
    for (int d = 1; d < C::DIMS; ++d) {
        T r[M];
        NodeIO<T, M>::load(ebuf + d * C::FSL + t * C::TSL + s * M, r);
#pragma unroll
        for (int v = 0; v < M; ++v) R[v] += ratio[d] * r[v];
    }
}

// EX: the variant that serves the guesses with more state -- the
// extrapolation of the previous predictor (guess 3) and the CERK guess
// (guess 4); solves with the other guesses use EX = false, which carries no
// code (or registers) for them.
template <class PDE, int DIM, int N, typename T, int TS, bool EX>
__global__ void __launch_bounds__(PredCfg<PDE, DIM, N, T, TS>::THREADS, PredCfg<PDE, DIM, N, T, TS>::MINB)
k_predictor(const KParams P)
{
    using C = PredCfg<PDE, DIM, N, T, TS>;
    constexpr int n = C::n, M = C::M, NS = C::NS, NF = C::NF, NREC = C::NREC;
    constexpr int EPB = C::EPB, RS = Geom<PDE, DIM, N>::RS;
    const Ops<T> &O = ops_of<T>(P);

    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sKw = reinterpret_cast<T *>(smem_raw);  // DIM x n x n (unscaled)
    T *sF0 = sKw + DIM * n * n;
    T *sF1 = sF0 + n;
    T *sDt = sF1 + n;                          // dt / dx_0 of the current tile
    T *sW = sDt + 1;                           // extrapolation weights [t][k] of the tile
    T *sIW = sW + n * n;                       // (dt / dx_0) iK1W of the tile
    const int tid = threadIdx.x;
    const bool act = tid < EPB * NS;
    const int g = act ? tid / NS : 0;
    const int s = act ? tid - g * NS : 0;
    const int tk = s / NF, pk = s - (s / NF) * NF;  // this thread's d-pencils
    const int tk0 = C::MAPB0 ? s % n : tk, pk0 = C::MAPB0 ? s / n : pk;  // its x-pencil
    T *ebuf = reinterpret_cast<T *>(smem_raw) + C::SHARED + g * C::ELEM;
    T *sQ = ebuf;                             // qbar[s][v]
    T *sFb = ebuf + NS * M;                   // Fbar[d][s][v]

    TcOp tcop{};
    if constexpr (C::TC) tcop = tc_operator<n>(reinterpret_cast<const float *>(O.Dm[0]));
    for (int i = tid; i < DIM * n * n; i += blockDim.x) sKw[i] = O.Kv[i / (n * n)][i % (n * n)];
    for (int i = tid; i < n; i += blockDim.x) {
        sF0[i] = O.F0[i];
        sF1[i] = O.F1[i];
    }
    __syncthreads();

    for (long long tile = blockIdx.x; tile < P.ntiles; tile += gridDim.x) {
        const int si = find_solve(P.solves, P.nsolves, tile, 0);
        const SolveDesc &S = P.solves[si];
        const double dt = solve_dt(P, S);
        if (!(dt > 0.0)) continue;  // uniform over the CTA: this solve takes no step
        if (tid == 0) sDt[0] = T(dt * S.inv_dx[0]);  // dt / dx_0 (see gather_R), read after a barrier
        // FP64: the time solve's operator scaled by dt / dx_0 (read after a
        // barrier), so that q[t] = u + sum_t' sIW[t][t'] R[t'] takes n FMAs per value
        if constexpr (sizeof(T) == 8)
            for (int i = tid; i < n * n; i += blockDim.x) sIW[i] = T(dt * S.inv_dx[0]) * O.iK1W[i];
        T idx[DIM], ratio[DIM];
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            if constexpr (sizeof(T) == 4) {
                idx[d] = S.inv_dx_f[d];
                ratio[d] = S.ratio_f[d];
            } else {
                idx[d] = S.inv_dx[d];
                ratio[d] = S.inv_dx[d] / S.inv_dx[0];
            }
        }

        const long long e = (tile - S.tile0_p) * EPB + g;
        const bool valid = act && e < S.E;
        const long long el = e < S.E ? e : S.E - 1;  // tail groups recompute the last element
        const long long ec = S.elist ? (long long)S.elist[el] : el;  // a listed subset of a block, or all
        // FP32 path: perturbations about the element's reference node
        typename PDE::template Ref<T> ref;
        double uref[M];
        T u[M];
        if constexpr (C::DELTA) {
#pragma unroll
            for (int v = 0; v < M; ++v) uref[v] = S.u[(ec * NS + C::SREF) * M + v];
            {
                T urf[M];
#pragma unroll
                for (int v = 0; v < M; ++v) urf[v] = narrow<T>(uref[v]);
                PDE::make_ref(P.pde, urf, ref);
            }
#pragma unroll
            for (int v = 0; v < M; ++v) u[v] = narrow<T>(S.u[(ec * NS + s) * M + v] - uref[v]);
        } else {
#pragma unroll
            for (int v = 0; v < M; ++v) u[v] = T(S.u[(ec * NS + s) * M + v]);
        }
        auto flx = [&](const T *qq, T(*FF)[M]) {
            if constexpr (C::DELTA) PDE::flux_delta(P.pde, ref, qq, FF);
            else PDE::flux(P.pde, qq, FF);
        };
        // the value whose d-derivative each direction needs: the flux F_d, or
        // for a purely non-conservative system the state itself
        auto xch = [&](const T *qq, T(*FF)[M]) {
            if constexpr (PDE::NCP) {
#pragma unroll
                for (int d = 0; d < DIM; ++d)
#pragma unroll
                    for (int v = 0; v < M; ++v) FF[d][v] = qq[v];
            } else {
                flx(qq, FF);
            }
        };
        // the absolute state of a node value (the FP32 path holds perturbations)
        auto absq = [&](const T *qq, T *qa) {
#pragma unroll
            for (int v = 0; v < M; ++v) {
                if constexpr (C::DELTA) qa[v] = qq[v] + ref.q[v];
                else qa[v] = qq[v];
            }
        };
        T dx0 = T(0);
        if constexpr (PDE::HAS_SRC) dx0 = T(1.0 / S.inv_dx[0]);
        // purely non-conservative system: -Dhat_d alpha at this node, once per
        // tile (alpha is constant in time), through ebuf's first NS words
        T gal[PDE::NCP ? DIM : 1];
        if constexpr (PDE::NCP) {
            if (act) ebuf[s] = u[PDE::IA];
            __syncthreads();
#pragma unroll
            for (int d = 0; d < DIM; ++d) {
                const int pd = ipow(n, d);
                const int kd = (s / pd) % n;
                const T *a = ebuf + (s - kd * pd);
                T acc = O.Dm[0][kd * n] * a[0];
#pragma unroll
                for (int j = 1; j < n; ++j) acc += O.Dm[0][kd * n + j] * a[j * pd];
                gal[d] = acc;
            }
            __syncthreads();  // ebuf is the exchange field from here on
        }
        // R = dx_0 L at (t, s) from the exchanged -Dhat_d derivatives in
        // ebuf: -sum_d (dx_0/dx_d) Dhat_d F_d, or -sum_d (dx_0/dx_d) B_d(q)
        // Dhat_d q; plus dx_0 S(q).  qq is this node's state at time level t.
        auto rhs = [&](int t, const T *qq, T *R) {
            if constexpr (PDE::NCP) {
                T qa[M];
                absq(qq, qa);
                const T ia = recip(qa[PDE::IA]), ir = recip(qa[PDE::IR]);
#pragma unroll
                for (int d = 0; d < DIM; ++d) {
                    T g[C::MX], b[M];
                    NodeIO<T, C::MX>::load(ebuf + d * C::FSL + t * C::TSL + s * C::MX, g);
                    PDE::bdot(qa, ia, ir, d, g, gal[d], b);
#pragma unroll
                    for (int v = 0; v < C::MR; ++v) R[v] = d == 0 ? b[v] : R[v] + ratio[d] * b[v];
                }
#pragma unroll
                for (int v = C::MR; v < M; ++v) R[v] = T(0);  // the material fields
            } else {
                gather_R<C, T>(ebuf, t, s, ratio, R);
            }
            if constexpr (PDE::HAS_SRC) {
                T qa[M], Sq[M];
                absq(qq, qa);
                PDE::source(P.pde, qa, Sq);
#pragma unroll
                for (int v = 0; v < M; ++v) R[v] += dx0 * Sq[v];
            }
        };

        // R(w) = dx_0 L(w) at this thread's spatial node for a time-constant
        // w: t = 0 pencils only (ebuf's t = 0 slice; free again when this
        // returns).  Every thread of the CTA calls it (barriers).
        auto spatial_R = [&](const T *w, T *R) {
            T F[DIM][M];
            xch(w, F);
            if (act) {
#pragma unroll
                for (int d = 0; d < DIM; ++d) NodeIO<T, C::MX>::store(ebuf + d * C::FSL + s * C::MX, F[d]);
            }
            __syncthreads();
            if (act)
                for (int item = s; item < DIM * NF * C::MX; item += NS) contract_item_t0<C, T>(ebuf, item, O.Dm[0]);
            __syncthreads();
            rhs(0, w, R);
            __syncthreads();
        };

        T q[n][M];
        int it0;  // Picard iterations already taken
        int P_it = S.picard;
        bool extrap = false;
        if constexpr (EX) extrap = S.guess == 3 && P.use_ctl_dt && S.ctl->dt_prev > 0.0;
        if (extrap) {
            // extrapolation of the previous step's predictor (Sec. 2.2):
            // q[t] = u + sum_k (L_k(1 + xi_t dt/dt_prev) - L_k(1)) qprev[k]
            if (tid == 0) extrap_weights<T, n>(O, T(dt / S.ctl->dt_prev), sW);
            __syncthreads();
            const T *qp = reinterpret_cast<const T *>(S.qprev) + ec * (n * NS * M);
#pragma unroll
            for (int t = 0; t < n; ++t)
#pragma unroll
                for (int v = 0; v < M; ++v) q[t][v] = u[v];
#pragma unroll 1
            for (int k = 0; k < n; ++k) {  // one previous time level at a time
                T qk[M];
                NodeIO<T, M>::load(qp + (k * NS + s) * M, qk);
#pragma unroll
                for (int t = 0; t < n; ++t) {
                    const T wk = sW[t * n + k];
#pragma unroll
                    for (int v = 0; v < M; ++v) q[t][v] += wk * qk[v];
                }
            }
            it0 = 0;
        } else {
            T R1[M];
            spatial_R(u, R1);
            const T dtT = sDt[0];
            if (S.guess == 3) P_it = S.picard_first;  // no previous predictor: the third-order guess
            if (S.guess == 2 || S.guess == 3) {
                // third-order guess (Sec. 2.2): q = u + tau k1 + tau^2 (k2 - k1) / (2 dt),
                // tau = xi dt, k1 = L(u), k2 = L(u + dt k1)
                T w[M], R2[M];
#pragma unroll
                for (int v = 0; v < M; ++v) w[v] = u[v] + dtT * R1[v];
                spatial_R(w, R2);
#pragma unroll
                for (int t = 0; t < n; ++t)
#pragma unroll
                    for (int v = 0; v < M; ++v)
                        q[t][v] = u[v] + dtT * (O.xi[t] * R1[v] + O.hxi2[t] * (R2[v] - R1[v]));
                it0 = 0;
            } else if (S.guess == 1) {
                // second-order guess: q = u + tau L(u)
#pragma unroll
                for (int t = 0; t < n; ++t)
#pragma unroll
                    for (int v = 0; v < M; ++v) q[t][v] = u[v] + dtT * (O.xi[t] * R1[v]);
                it0 = 0;
            } else if (EX && S.guess == 4) {
                if constexpr (EX) {
                    // CERK guess (Sec. 2.2): q = u + dt sum_i b_i(xi) k_i with
                    // k_i = L(u + dt sum_{j<i} a_ij k_j), the scheme of
                    // cerk_stages(N) stages (Ops::ck_a, ck_b); accumulated stage
                    // by stage
                    constexpr int CS = cerk_stages(N);
                    T w[M], Rk[M];
#pragma unroll
                    for (int t = 0; t < n; ++t)
#pragma unroll
                        for (int v = 0; v < M; ++v) q[t][v] = u[v] + dtT * (O.ck_b[0][t] * R1[v]);
                    if constexpr (CS == 4) {
                        // the classical method: each stage state from the previous k
#pragma unroll
                        for (int v = 0; v < M; ++v) w[v] = u[v] + T(0.5) * dtT * R1[v];
#pragma unroll 1
                        for (int st = 1; st < 4; ++st) {
                            spatial_R(w, Rk);
#pragma unroll
                            for (int t = 0; t < n; ++t) {
                                const T bt = st == 3 ? O.ck_b[3][t] : O.ck_b[1][t];  // b2 = b3
#pragma unroll
                                for (int v = 0; v < M; ++v) q[t][v] += dtT * (bt * Rk[v]);
                            }
                            const T cs = st == 1 ? T(0.5) : T(1);
#pragma unroll
                            for (int v = 0; v < M; ++v) w[v] = u[v] + cs * dtT * Rk[v];
                        }
                    } else {
                        // the earlier stages' k of this thread's node wait in the
                        // exchange field's time slices t >= 1 (only the t = 0
                        // slices serve the L evaluations); the variables past MX
                        // have k = 0
                        static_assert(CS - 1 <= DIM * (n - 1), "CERK stage slots");
                        auto kslot = [&](int j) {
                            return ebuf + (j / (n - 1)) * C::FSL + (1 + j % (n - 1)) * C::TSL + s * C::MX;
                        };
                        if (act) NodeIO<T, C::MX>::store(kslot(0), R1);
#pragma unroll 1
                        for (int st = 1; st < CS; ++st) {
#pragma unroll
                            for (int v = 0; v < M; ++v) w[v] = T(0);
#pragma unroll 1
                            for (int j = 0; j < st; ++j) {
                                T kj[C::MX];
                                NodeIO<T, C::MX>::load(kslot(j), kj);
                                const T a = O.ck_a[st * (st - 1) / 2 + j];
#pragma unroll
                                for (int v = 0; v < C::MX; ++v) w[v] += a * kj[v];
                            }
#pragma unroll
                            for (int v = 0; v < M; ++v) w[v] = u[v] + dtT * w[v];
                            spatial_R(w, Rk);
#pragma unroll
                            for (int t = 0; t < n; ++t) {
                                const T bt = O.ck_b[st][t];
#pragma unroll
                                for (int v = 0; v < M; ++v) q[t][v] += dtT * (bt * Rk[v]);
                            }
                            if (act && st < CS - 1) NodeIO<T, C::MX>::store(kslot(st), Rk);
                        }
                    }
                }
                it0 = 0;
            } else {
                // trivial guess q = u: its first Picard iteration, taken on
                // the time-constant q (one flux per spatial node)
#pragma unroll
                for (int t = 0; t < n; ++t)
#pragma unroll
                    for (int v = 0; v < M; ++v) q[t][v] = u[v] + dtT * (O.c1[t] * R1[v]);
                it0 = 1;
            }
        }
        // ---- Picard iterations of eq. pde.st2 ------------------------------
        for (int it = it0; it < P_it; ++it) {
            if constexpr (C::QX) {
                // the state through shared memory; each pencil owner forms its F_d
                if (act) {
#pragma unroll
                    for (int t = 0; t < n; ++t) NodeIO<T, M>::store(ebuf + DIM * C::FSL + t * C::TSL + s * M, q[t]);
                }
                __syncthreads();
                if (act) contract_all_qx<C, T>(ebuf, tk0, pk0, tk, pk, O, flx);
            } else {
#pragma unroll
                for (int t = 0; t < n; ++t) {
                    T F[DIM][M];
                    xch(q[t], F);
                    if (act) {
#pragma unroll
                        for (int d = 0; d < DIM; ++d)
                            NodeIO<T, C::MX>::store(ebuf + d * C::FSL + t * C::TSL + s * C::MX, F[d]);
                    }
                }
                __syncthreads();
                if constexpr (C::TC) contract_all_mma<C>(reinterpret_cast<float *>(smem_raw) + C::SHARED, tcop);
                else if (act) contract_all<C, T>(ebuf, tk0, pk0, tk, pk, O);
            }
            __syncthreads();
            {
                T R[n][M];
#pragma unroll
                for (int t = 0; t < n; ++t) rhs(t, q[t], R[t]);
                // FP64: the scaled operator from shared memory, n FMAs per value
                // (the FP64 pipe bounds the kernel: 8 % faster than the
                // constant-bank operator times dt/dx_0); FP32: the constant-bank
                // operator (shared-memory bandwidth bounds that kernel)
#pragma unroll
                for (int v = 0; v < C::MR; ++v)  // rows MR.. have R = 0: q stays u there
#pragma unroll
                    for (int t = 0; t < n; ++t) {
                        if constexpr (sizeof(T) == 8) {
                            T acc = u[v];
#pragma unroll
                            for (int tp = 0; tp < n; ++tp) acc += sIW[t * n + tp] * R[tp][v];
                            q[t][v] = acc;
                        } else {
                            T acc = O.iK1W[t * n] * R[0][v];
#pragma unroll
                            for (int tp = 1; tp < n; ++tp) acc += O.iK1W[t * n + tp] * R[tp][v];
                            q[t][v] = u[v] + sDt[0] * acc;
                        }
                    }
            }
            __syncthreads();
        }

        if constexpr (EX) {
            if (S.guess == 3 && valid) {  // this step's predictor, for the next step's guess
                T *qp = reinterpret_cast<T *>(S.qprev) + ec * (n * NS * M);
#pragma unroll
                for (int t = 0; t < n; ++t) NodeIO<T, M>::store(qp + (t * NS + s) * M, q[t]);
            }
        }

        // ---- time averages qbar, Fbar_d (registers) ------------------------
        T qb[M], Fb[DIM][M];
#pragma unroll
        for (int v = 0; v < M; ++v) {
            qb[v] = T(0);
#pragma unroll
            for (int d = 0; d < DIM; ++d) Fb[d][v] = T(0);
        }
#pragma unroll
        for (int t = 0; t < n; ++t) {
            const T wt = O.w[t];
#pragma unroll
            for (int v = 0; v < M; ++v) qb[v] += wt * q[t][v];
            if constexpr (!PDE::NCP) {
                T F[DIM][M];
                flx(q[t], F);
#pragma unroll
                for (int v = 0; v < M; ++v)
#pragma unroll
                    for (int d = 0; d < DIM; ++d) Fb[d][v] += wt * F[d][v];
            }
        }
        // purely non-conservative system: the volume integrals of B(q) grad q
        // at the time nodes average to their value at qbar (B(q) g is linear
        // in the evolved variables, the material fields are constant in time):
        // V = L(qbar), one more evaluation on the time-constant qbar
        T Vnc[M];
        if constexpr (PDE::NCP) spatial_R(qb, Vnc);
        if (act) {
            NodeIO<T, M>::store(sQ + s * M, qb);
            if constexpr (!PDE::NCP) {
#pragma unroll
                for (int d = 0; d < DIM; ++d) NodeIO<T, M>::store(sFb + (d * NS + s) * M, Fb[d]);
            }
        }
        __syncthreads();

        // ---- volume term V = sum_d (1/dx_d) Kw Fbar_d + S(qbar) -------------
        if constexpr (PDE::NCP) {
            if (valid) {
                T *Vout = reinterpret_cast<T *>(S.V) + ec * (NS * M);
#pragma unroll
                for (int v = 0; v < M; ++v) Vout[s * M + v] = idx[0] * Vnc[v];
            }
        } else if (valid) {
            T *Vout = reinterpret_cast<T *>(S.V) + ec * (NS * M);
            int kd[DIM];
            {
                int r = s;
#pragma unroll
                for (int d = 0; d < DIM; ++d) { kd[d] = r % n; r /= n; }
            }
            T Vn[M];
#pragma unroll
            for (int v = 0; v < M; ++v) Vn[v] = T(0);
#pragma unroll
            for (int d = 0; d < DIM; ++d) {
                const int pd = ipow(n, d);
                const int base = s - kd[d] * pd;
                const T *Krow = sKw + (d * n + kd[d]) * n;
                T a[M];
#pragma unroll
                for (int v = 0; v < M; ++v) a[v] = T(0);
#pragma unroll
                for (int j = 0; j < n; ++j) {
                    T f[M];
                    NodeIO<T, M>::load(sFb + (d * NS + base + j * pd) * M, f);
#pragma unroll
                    for (int v = 0; v < M; ++v) a[v] += Krow[j] * f[v];
                }
#pragma unroll
                for (int v = 0; v < M; ++v) Vn[v] += idx[d] * a[v];
            }
            if constexpr (PDE::HAS_SRC) {  // S linear: its time average is S(qbar)
                T qa[M], Sq[M];
                absq(qb, qa);
                PDE::source(P.pde, qa, Sq);
#pragma unroll
                for (int v = 0; v < M; ++v) Vn[v] += Sq[v];
            }
#pragma unroll
            for (int v = 0; v < M; ++v) Vout[s * M + v] = Vn[v];
        }

        // ---- face traces of the time averages and their wave speeds --------
        T *trE = reinterpret_cast<T *>(S.tr) + ec * (NREC * RS);
        if constexpr (NREC <= NS) {
            // one record (all variables) per thread; wave speed in place
            if (valid) {
                for (int rec = s; rec < NREC; rec += NS) {
                    const int d = rec / (2 * NF);
                    const int side = (rec / NF) & 1;
                    const int p = rec - (rec / NF) * NF;
                    const int pd = d == 0 ? 1 : (d == 1 ? n : n * n);
                    const int s0 = (p % pd) + (p / pd) * pd * n;
                    const T *phi = side ? sF1 : sF0;
                    T aq[M], af[M];
#pragma unroll
                    for (int v = 0; v < M; ++v) { aq[v] = T(0); af[v] = T(0); }
#pragma unroll
                    for (int j = 0; j < n; ++j) {
                        T qj[M];
                        NodeIO<T, M>::load(sQ + (s0 + j * pd) * M, qj);
                        const T pj = phi[j];
#pragma unroll
                        for (int v = 0; v < M; ++v) aq[v] += pj * qj[v];
                        if constexpr (!PDE::NCP) {
                            T fj[M];
                            NodeIO<T, M>::load(sFb + (d * NS + s0 + j * pd) * M, fj);
#pragma unroll
                            for (int v = 0; v < M; ++v) af[v] += pj * fj[v];
                        }
                    }
                    T *r = trE + rec * RS;
                    T full[M];
                    absq(aq, full);
#pragma unroll
                    for (int v = 0; v < M; ++v) {
                        r[v] = aq[v];
                        if constexpr (!PDE::NCP) r[M + v] = af[v];
                    }
                    r[C::LAM] = PDE::max_eig(P.pde, full, d);
                    if constexpr (RS > C::LAM + 1) r[C::LAM + 1] = T(0);
                }
            }
        } else {
            // more records than threads: (record, variable) items, then the
            // wave speeds from the stashed face states
            T *sStash = ebuf + (1 + DIM) * NS * M;
            if (act) {
                for (int i = s; i < NREC * M; i += NS) {
                    const int rec = i / M, v = i - rec * M;
                    const int d = rec / (2 * NF);
                    const int side = (rec / NF) & 1;
                    const int p = rec - (rec / NF) * NF;
                    const int pd = ipow(n, d);
                    const int s0 = (p % pd) + (p / pd) * pd * n;
                    const T *phi = side ? sF1 : sF0;
                    T aq = T(0), af = T(0);
#pragma unroll
                    for (int j = 0; j < n; ++j) {
                        aq += phi[j] * sQ[(s0 + j * pd) * M + v];
                        if constexpr (!PDE::NCP) af += phi[j] * sFb[(d * NS + s0 + j * pd) * M + v];
                    }
                    sStash[rec * M + v] = aq;
                    if (valid) {
                        trE[rec * RS + v] = aq;
                        if constexpr (!PDE::NCP) trE[rec * RS + M + v] = af;
                    }
                }
            }
            __syncthreads();
            if (valid) {
                for (int rec = s; rec < NREC; rec += NS) {
                    const int d = rec / (2 * NF);
                    T full[M];
                    absq(sStash + rec * M, full);
                    trE[rec * RS + C::LAM] = PDE::max_eig(P.pde, full, d);
                    if constexpr (RS > C::LAM + 1) trE[rec * RS + C::LAM + 1] = T(0);
                }
            }
        }
        if constexpr (C::DELTA) {
            if (valid && s == 0) {  // the reference state, kept in FP64 for the corrector
#pragma unroll
                for (int v = 0; v < M; ++v) S.ref[ec * C::RF + v] = uref[v];
            }
        }
        __syncthreads();  // ebuf is reused by the next tile
    }
}

#include "predictor_xt.cuh"

// ===========================================================================
// Corrector
// ===========================================================================

// A CTA takes a tile of EPB consecutive elements.  All its inputs -- its own
// trace records (one contiguous range), the 2d neighbour face chunks of
// every element, u^n and V -- are staged into shared memory with cp.async
// first (every load in flight at once), then: Rusanov flux per (element,
// face record), all variables; per (element, node): lift, FP64 update with
// vector stores and the wave speeds of the new state from registers; one
// atomic per CTA for the maxima.

__device__ __forceinline__ void cp_async(void *dst, const void *src, int bytes)
{
    const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(dst));
    if (bytes == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(src));
    else if (bytes == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(src));
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(src));
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }

__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// wait for every committed group of this thread's copies but the latest
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

template <int GRAN>
__device__ __forceinline__ void stage(void *dst, const void *src, int bytes, int tid, int nthr)
{
    const int units = bytes / GRAN;
    unsigned char *d = static_cast<unsigned char *>(dst);
    const unsigned char *s = static_cast<const unsigned char *>(src);
    for (int i = tid; i < units; i += nthr) cp_async(d + i * GRAN, s + i * GRAN, GRAN);
}

template <class PDE, int DIM, int N, typename T, int TS = 0>
struct CorrCfg {
    using G = Geom<PDE, DIM, N>;
    static constexpr int n = G::n, M = G::M, NS = G::NS, NF = G::NF, NREC = G::NREC, RS = G::RS;
    static constexpr size_t OWN = sizeof(T) * NREC * RS;          // per element
    static constexpr size_t NB = sizeof(T) * 2 * DIM * NF * RS;   // per element
    static constexpr size_t UB = sizeof(double) * NS * M;
    static constexpr size_t VB = sizeof(T) * NS * M;
    static constexpr size_t FS = sizeof(T) * NREC * M;
    // u^n and V are staged in shared memory, except on the FP64 path when an
    // element's staged inputs are large (3D elasticity: 43 KB per element):
    // there the update reads them from global memory once, and the smaller
    // footprint lets more CTAs share an SM (corrector 7.8 -> 7.2 ms at 64^3,
    // N = 3; the FP32 path measured slower without the staging)
    static constexpr bool STAGE_UV =
        sizeof(T) == 4 || align16(OWN) + align16(NB) + align16(UB) + align16(VB) <= 8192;
    static constexpr size_t PER_ELEM =
        align16(OWN) + align16(NB) + (STAGE_UV ? align16(UB) + align16(VB) : 0) + align16(FS);
    // shapes 0, 1, 2, 4: 256-, 128-, 512- and 64-thread CTAs; shape 3: every
    // warp takes one element of the tile on its own (its own shared-memory
    // slice, warp-level synchronisation only), NW warps per CTA; shape 5:
    // 128-thread CTAs whose tile is SUB consecutive groups of EPB elements,
    // the next group's inputs staged (double-buffered) while the current
    // group is computed
    static constexpr bool WM = TS == 3;
    static constexpr int SUB = TS == 5 ? 4 : 1;
    static constexpr int BUF = SUB > 1 ? 2 : 1;
    static constexpr int THREADS_CTA = (TS == 1 || TS == 5) ? 128 : (TS == 2 ? 512 : (TS == 4 ? 64 : 256));
    static constexpr int EPB_T = cmax(1, THREADS_CTA / NS);
    static constexpr size_t STAGED = align16(OWN) + align16(NB) + (STAGE_UV ? align16(UB) + align16(VB) : 0);
    static constexpr int EPB_S = cmax(1, (int)((110 * 1024) / (PER_ELEM + (BUF - 1) * STAGED)));
    static constexpr int EPB = WM ? 1 : cmin(EPB_T, EPB_S);  // elements per shared-memory unit (group)
    // one staging buffer (the group's own records, neighbour chunks, u^n, V);
    // BUF of them, PB bytes apart
    static constexpr size_t O_OWN = 0;
    static constexpr size_t O_NB = align16(EPB * OWN);
    static constexpr size_t O_U = O_NB + align16(EPB * NB);
    static constexpr size_t O_V = O_U + (STAGE_UV ? align16(EPB * UB) : 0);
    static constexpr size_t PB = O_V + (STAGE_UV ? align16(EPB * VB) : 0);
    static constexpr size_t O_FS = BUF * PB;
    static constexpr size_t O_LIFT = O_FS + align16(EPB * FS);
    static constexpr size_t O_DEL = O_LIFT + align16(sizeof(T) * 2 * 3 * NMAX);
    static constexpr bool DELTA = sizeof(T) == 4;
    static constexpr int RF = M;
    static constexpr int LAM = G::LAM;
    // FP32 path of a non-conservative system: each element's reference in T
    // (the path integral needs absolute face states)
    static constexpr size_t O_REFO = O_DEL + (DELTA ? align16(sizeof(T) * EPB * 2 * DIM * 2 * M) : 0);
    static constexpr size_t O_RED = O_REFO + (DELTA && PDE::NCP ? align16(sizeof(T) * EPB * M) : 0);
    // the CTA reduction: 16 warps x 4 values, then 16 flags
    static constexpr size_t BYTES = O_RED + 64 * sizeof(double) + 16 * sizeof(int);  // one unit (the CTA, or a warp)
    static constexpr int NW = WM ? cmax(1, cmin(8, (int)((200 * 1024) / BYTES))) : 1;
    static constexpr int THREADS = WM ? 32 * NW : THREADS_CTA;
    static constexpr int EPB_TILE = WM ? NW : EPB * SUB;  // elements per tile of the launch
    static constexpr size_t CTA_BYTES = NW * BYTES;
    static_assert(CTA_BYTES <= 227 * 1024, "corrector shared memory");
    // copy granules (bytes): the largest of 16/8/4 dividing offsets and sizes
    static constexpr int G_OWN = cgcd((int)OWN, 16);
    static constexpr int G_NB = cgcd((int)(sizeof(T) * RS), 16);
    static constexpr int G_U = cgcd((int)UB, 16);
    static constexpr int G_V = cgcd((int)VB, 16);
};

// neighbour of element e of solve S (x-fastest numbering over S.cells)
// along d, periodic; the divisions by the cell counts are multiply-highs
__device__ __forceinline__ int neighbour_of(const SolveDesc &S, int e, int d, int off)
{
    const int cx = S.cells[0], cy = S.cells[1], cz = S.cells[2];
    const unsigned q0 = fdiv((unsigned)e, S.div_cx), q1 = fdiv(q0, S.div_cy);
    int ix = e - (int)q0 * cx, iy = (int)(q0 - q1 * (unsigned)cy), iz = (int)q1;
    if (d == 0) ix = ix + off < 0 ? cx - 1 : (ix + off >= cx ? 0 : ix + off);
    else if (d == 1) iy = iy + off < 0 ? cy - 1 : (iy + off >= cy ? 0 : iy + off);
    else iz = iz + off < 0 ? cz - 1 : (iz + off >= cz ? 0 : iz + off);
    return ix + cx * (iy + cy * iz);
}

// Neighbour of element e (at cell (ix, iy, iz); no divisions) of a block
// across its face (d, side): the block element (>= 0, periodic), or -(1 + j)
// for chunk j of the halo that another block of a partitioned mesh filled
// (j: the element's index over the other directions, lowest fastest).  Sg
// is the descriptor in device memory (its halo pointers are read with
// runtime indices).
__device__ __forceinline__ int neighbour_or_halo_at(int e, int ix, int iy, int iz, const SolveDesc *Sg, int cx, int cy,
                                                    int cz, int d, int side)
{
    const int k = d == 0 ? ix : (d == 1 ? iy : iz);
    const int cd = d == 0 ? cx : (d == 1 ? cy : cz);
    const int stride = d == 0 ? 1 : (d == 1 ? cx : cx * cy);
    const bool edge = side ? k == cd - 1 : k == 0;
    if (edge && Sg->halo_tr[d][side] != nullptr)
        return -1 - (d == 0 ? iy + cy * iz : (d == 1 ? ix + cx * iz : ix + cx * iy));
    if (edge) return side ? e - (cd - 1) * stride : e + (cd - 1) * stride;  // periodic
    return side ? e + stride : e - stride;
}

template <class PDE, int DIM, int N, typename T, int TS>
__global__ void __launch_bounds__(CorrCfg<PDE, DIM, N, T, TS>::THREADS)
k_corrector(const KParams P)
{
    using C = CorrCfg<PDE, DIM, N, T, TS>;
    constexpr int n = C::n, M = C::M, NS = C::NS, NF = C::NF, NREC = C::NREC, RS = C::RS;
    constexpr int EPT = C::EPB_TILE;

    // the unit that shares a shared-memory slice and synchronises: the CTA,
    // or (shape 3) each warp with its own slice and element
    const int wid = threadIdx.x >> 5;
    const int tid = C::WM ? (int)(threadIdx.x & 31) : (int)threadIdx.x;
    const int nthr = C::WM ? 32 : (int)blockDim.x;
    auto usync = [&]() {
        if constexpr (C::WM) __syncwarp();
        else __syncthreads();
    };
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char *sb = smem_raw + (C::WM ? wid * C::BYTES : 0);
    // staging buffer b (BUF of them): the group's own records, neighbour
    // chunks, u^n and V
    auto own_of = [&](int b) { return reinterpret_cast<T *>(sb + (size_t)b * C::PB + C::O_OWN); };
    auto nbr_of = [&](int b) { return reinterpret_cast<T *>(sb + (size_t)b * C::PB + C::O_NB); };
    auto u_of = [&](int b) { return reinterpret_cast<double *>(sb + (size_t)b * C::PB + C::O_U); };
    auto v_of = [&](int b) { return reinterpret_cast<T *>(sb + (size_t)b * C::PB + C::O_V); };
    T *sFs = reinterpret_cast<T *>(sb + C::O_FS);
    T *sL = reinterpret_cast<T *>(sb + C::O_LIFT);  // [side][d][k]
    T *sDel = reinterpret_cast<T *>(sb + C::O_DEL);  // [el][d][side][dF | dq][M]
    T *sRefO = reinterpret_cast<T *>(sb + C::O_REFO);  // [el][M]
    double *red = reinterpret_cast<double *>(sb + C::O_RED);
    // shape 3: each lane's wave-speed maxima and non-finite flag, gathered
    // over the warp's elements of one solve and flushed when the solve changes
    T acc_l[DIM];
#pragma unroll
    for (int d = 0; d < DIM; ++d) acc_l[d] = T(0);
    bool acc_bad = false;
    Control *acc_ctl = nullptr;
    auto flush = [&]() {  // warp-uniform
        if (acc_ctl == nullptr) return;
        const unsigned anyb = __any_sync(0xffffffffu, acc_bad);
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            T x = acc_l[d];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const T y = __shfl_xor_sync(0xffffffffu, x, o);
                x = y > x ? y : x;
            }
            if ((threadIdx.x & 31) == 0)
                atomicMax(&acc_ctl->lam_acc[d], (unsigned long long)__double_as_longlong(double(x)));
            acc_l[d] = T(0);
        }
        if ((threadIdx.x & 31) == 0 && anyb) atomicOr(&acc_ctl->flags, FLAG_NONFINITE);
        acc_bad = false;
    };

    for (long long tile = blockIdx.x; tile < P.ntiles; tile += gridDim.x) {
        const int si = find_solve(P.solves, P.nsolves, tile, 1);
        const SolveDesc S = P.solves[si];
        const double dt = solve_dt(P, S);
        if (!(dt > 0.0)) continue;  // uniform over the CTA

        const int et = (int)((tile - S.tile0_c) * EPT);              // the tile's first element
        const int nt = (S.E - et) < EPT ? (int)(S.E - et) : EPT;     // and its element count
        if (C::WM && wid >= nt) continue;  // uniform over the warp
        const T *tr = reinterpret_cast<const T *>(S.tr);

        // neighbour (block element, or halo chunk) across face c = (el, d,
        // side) of the group that starts at element e0g in cell c0: carries
        // per element from the group's first cell
        const int cx = S.cells[0], cy = S.cells[1], cz = S.cells[2];
        struct Cell {
            int x, y, z;
        };
        auto cell_of = [&](int e) {  // by multiply-high divisions
            const unsigned q0 = fdiv((unsigned)e, S.div_cx), q1 = fdiv(q0, S.div_cy);
            return Cell{e - (int)q0 * cx, (int)(q0 - q1 * (unsigned)cy), (int)q1};
        };
        auto nb_of = [&](int e0g, Cell c0, int c) {
            const int el = c / (2 * DIM), d = (c / 2) % DIM, side = c & 1;
            int ix = c0.x + el, iy = c0.y, iz = c0.z;
            while (ix >= cx) {  // el < EPB: a few rows at most
                ix -= cx;
                if (++iy == cy) {
                    iy = 0;
                    ++iz;
                }
            }
            return neighbour_or_halo_at(e0g + el, ix, iy, iz, P.solves + si, cx, cy, cz, d, side);
        };
        for (int i = tid; i < DIM * n; i += nthr) {
            const int d = i / n, k = i % n;
            if constexpr (sizeof(T) == 4) {  // precomputed on the host: no FP64 work here
                sL[(0 * 3 + d) * NMAX + k] = P.solves[si].lift_f[0][d][k];
                sL[(1 * 3 + d) * NMAX + k] = P.solves[si].lift_f[1][d][k];
            } else {
                const double idx = P.solves[si].inv_dx[d];  // runtime index: read from global
                sL[(0 * 3 + d) * NMAX + k] = T(idx * P.b.inv_w[k] * P.b.F0[k]);
                sL[(1 * 3 + d) * NMAX + k] = T(idx * P.b.inv_w[k] * P.b.F1[k]);
            }
        }

        // the tile is ngrp groups of EPB elements (one group but for shape 5);
        // group g is staged into buffer g % BUF, the next one while g is
        // computed; the staging is one round of loads (the neighbour indices
        // are formed where they are used, not published through a barrier)
        const int ngrp = (C::WM || C::SUB == 1) ? 1 : (nt + C::EPB - 1) / C::EPB;
        auto grp_e0 = [&](int g) { return C::WM ? et + wid : (C::SUB == 1 ? et : et + g * C::EPB); };
        auto grp_ne = [&](int g) {
            return C::WM ? 1 : (C::SUB == 1 ? nt : (nt - g * C::EPB < C::EPB ? nt - g * C::EPB : C::EPB));
        };
        auto stage_group = [&](int g, int b, const Cell &c0) {  // c0: the group's first cell
            const int e0 = grp_e0(g), ne = grp_ne(g);
            T *sNb = nbr_of(b);
            stage<C::G_OWN>(own_of(b), tr + (long long)e0 * NREC * RS, ne * (int)C::OWN, tid, nthr);
            if constexpr (C::STAGE_UV) {
                stage<C::G_U>(u_of(b), S.u + (long long)e0 * NS * M, ne * (int)C::UB, tid, nthr);
                stage<C::G_V>(v_of(b), reinterpret_cast<const T *>(S.V) + (long long)e0 * NS * M, ne * (int)C::VB,
                              tid, nthr);
            }
            {
                // the neighbour chunks: tpc consecutive threads per chunk (element,
                // d, side), which forms its neighbour index once; ng = nthr / tpc
                // >= nch groups whenever tpc > 1, so every chunk has one group
                constexpr int units = (int)(sizeof(T) * NF * RS) / C::G_NB;
                const int nch = ne * 2 * DIM;
                const int tpc = nthr >= 2 * nch ? nthr / nch : 1;
                const int ng = nthr / tpc;
                for (int c = tid / tpc; c < nch && tid < ng * tpc; c += ng) {
                    const int d = (c / 2) % DIM;
                    const int side = c & 1;
                    const int nb = nb_of(e0, c0, c);
                    const T *src = nb >= 0 ? tr + (((long long)nb * DIM + d) * 2 + (1 - side)) * NF * RS
                                           : reinterpret_cast<const T *>(P.solves[si].halo_tr[d][side]) +
                                                 (long long)(-1 - nb) * NF * RS;
                    unsigned char *dst = reinterpret_cast<unsigned char *>(sNb + (size_t)c * NF * RS);
                    for (int u_ = tid % tpc; u_ < units; u_ += tpc)
                        cp_async(dst + u_ * C::G_NB, reinterpret_cast<const unsigned char *>(src) + u_ * C::G_NB,
                                 C::G_NB);
                }
            }
        };

        T lmax[DIM];
#pragma unroll
        for (int d = 0; d < DIM; ++d) lmax[d] = T(0);
        bool bad = false;
        Cell cg = cell_of(grp_e0(0));
        stage_group(0, 0, cg);
        if constexpr (C::BUF > 1) cp_async_commit();
        for (int g = 0; g < ngrp; ++g) {
            const int b = C::BUF > 1 ? (g & 1) : 0;
            const Cell c0 = cg;  // this group's first cell
            if constexpr (C::BUF > 1) {
                if (g + 1 < ngrp) {
                    cg = cell_of(grp_e0(g + 1));
                    stage_group(g + 1, b ^ 1, cg);
                }
                cp_async_commit();  // (an empty group when nothing was staged)
            }
            const int e0 = grp_e0(g), ne = grp_ne(g);
            const T *sOwn = own_of(b), *sNb = nbr_of(b);
            const double *sU = u_of(b);
            const T *sV = v_of(b);
            if constexpr (C::DELTA) {
                // reference differences across every face, sign +1 on the
                // xi_d = 1 face and -1 on the xi_d = 0 face:  dq = q_ref(nb) -
                // q_ref(own) formed in FP64 and rounded (it is O(h)), and
                // dF = F_d(q_ref(nb)) - F_d(q_ref(own)) by the perturbation flux
                for (int c = tid; c < ne * 2 * DIM; c += nthr) {
                    const int el = c / (2 * DIM), d = (c / 2) % DIM, side = c & 1;
                    const double *ro = S.ref + (long long)(e0 + el) * C::RF;
                    const int nb = nb_of(e0, c0, c);
                    const double *rn = nb >= 0 ? S.ref + (long long)nb * C::RF
                                               : P.solves[si].halo_ref[d][side] + (long long)(-1 - nb) * C::RF;
                    double qo[M];
                    T dq[M];
#pragma unroll
                    for (int v = 0; v < M; ++v) {
                        qo[v] = ro[v];
                        dq[v] = narrow<T>(rn[v] - qo[v]);
                    }
                    typename PDE::template Ref<T> rr;
                    {
                        T qf[M];
#pragma unroll
                        for (int v = 0; v < M; ++v) qf[v] = narrow<T>(qo[v]);
                        PDE::make_ref(P.pde, qf, rr);
                        if constexpr (PDE::NCP) {
                            if (d == 0 && side == 0) {
#pragma unroll
                                for (int v = 0; v < M; ++v) sRefO[el * M + v] = qf[v];
                            }
                        }
                    }
                    T dF[DIM][M];
                    PDE::flux_delta(P.pde, rr, dq, dF);
                    const T sg = side ? T(1) : T(-1);
#pragma unroll
                    for (int v = 0; v < M; ++v) {
                        T f = dF[0][v];
#pragma unroll
                        for (int k = 1; k < DIM; ++k) f = d == k ? dF[k][v] : f;
                        sDel[(c * 2 + 0) * M + v] = sg * f;
                        sDel[(c * 2 + 1) * M + v] = sg * dq[v];
                    }
                }
            }
            if constexpr (C::BUF > 1) cp_async_wait_prev();  // this group's copies (all but the latest group)
            else cp_async_wait_all();
            usync();

            // ---- Rusanov flux per (element, face record), all variables --------
            for (int i = tid; i < ne * NREC; i += nthr) {
                const int el = i / NREC;
                const int rec = i - el * NREC;
                const int d = rec / (2 * NF);
                const int side = (rec / NF) & 1;
                const int p = rec - (rec / NF) * NF;
                const T *own = sOwn + (el * NREC + rec) * RS;
                const T *nb = sNb + ((size_t)(el * DIM + d) * 2 + side) * NF * RS + p * RS;
                const T *L = side ? own : nb;
                const T *R = side ? nb : own;
                const T smax = tmax(L[C::LAM], R[C::LAM]);
                const T *dl = sDel + ((((el * DIM + d) * 2 + side) * 2) * M);
                T f[M];
                if constexpr (PDE::NCP) {
                    // path-conservative Rusanov (eq. pc.scheme, eq. rusanov): the
                    // lower element (side 1) receives -Theta dq/2 + J/2, the upper
                    // one -Theta dq/2 - J/2; Theta = s_max on the evolved variables
                    // only (the material fields obey q_t = 0)
                    T dq[M], qa[M], J[M];
#pragma unroll
                    for (int v = 0; v < M; ++v) {
                        dq[v] = R[v] - L[v];
                        qa[v] = L[v];
                        if constexpr (C::DELTA) {
                            // perturbations about each element's own reference
                            dq[v] += dl[M + v];
                            qa[v] += sRefO[el * M + v] - (side ? T(0) : dl[M + v]);
                        }
                    }
                    PDE::path_jump(qa, dq, d, J);
                    const T hs = side ? T(0.5) : T(-0.5);
#pragma unroll
                    for (int v = 0; v < M; ++v) f[v] = v < PDE::MEV ? hs * J[v] - T(0.5) * smax * dq[v] : T(0);
                } else {
#pragma unroll
                    for (int v = 0; v < M; ++v) {
                        f[v] = T(0.5) * (L[M + v] + R[M + v]) - T(0.5) * smax * (R[v] - L[v]);
                        if constexpr (C::DELTA) {
                            // traces are perturbations about each element's own reference:
                            // add the reference part of the Rusanov flux minus own F_ref
                            f[v] += (side ? T(0.5) : T(-0.5)) * dl[v] - T(0.5) * smax * dl[M + v];
                        }
                    }
                }
#pragma unroll
                for (int v = 0; v < M; ++v) sFs[(el * NREC + rec) * M + v] = f[v];
            }
            usync();

            // ---- per node: surface lift, update u^{n+1} = u^n + dt (V - surface),
            // ---- then the wave speeds of u^{n+1} and the non-finite check -------
            // (wave speeds in the compute type T; only the per-CTA maxima are widened)
            double *uo = S.u_out + (long long)e0 * NS * M;
            for (int i = tid; i < ne * NS; i += nthr) {
                const int el = i / NS;
                const int sn = i - el * NS;
                int kk[DIM], pp[DIM];
                {
                    int rr = sn;
#pragma unroll
                    for (int d = 0; d < DIM; ++d) {
                        kk[d] = rr % n;
                        rr /= n;
                        const int pd = ipow(n, d);
                        pp[d] = (sn % pd) + (sn / (pd * n)) * pd;
                    }
                }
                double un[M];
                T vn[M], qs[M];
                if constexpr (C::STAGE_UV) {
                    NodeIO<double, M>::load(sU + i * M, un);
                    NodeIO<T, M>::load(sV + i * M, vn);
                } else {
                    NodeIO<double, M>::load(S.u + ((long long)e0 * NS + i) * M, un);
                    NodeIO<T, M>::load(reinterpret_cast<const T *>(S.V) + ((long long)e0 * NS + i) * M, vn);
                }
#pragma unroll
                for (int v = 0; v < M; ++v) {
                    T surf = T(0);
#pragma unroll
                    for (int d = 0; d < DIM; ++d) {
                        const T fp = sFs[(el * NREC + (d * 2 + 1) * NF + pp[d]) * M + v];
                        const T fm = sFs[(el * NREC + (d * 2 + 0) * NF + pp[d]) * M + v];
                        surf += sL[(3 + d) * NMAX + kk[d]] * fp - sL[d * NMAX + kk[d]] * fm;
                    }
                    un[v] = un[v] + dt * widen<T>(vn[v] - surf);
                    bad |= dbl_nonfinite(un[v]);
                    qs[v] = narrow<T>(un[v]);
                }
                NodeIO<double, M>::store(uo + i * M, un);
#pragma unroll
                for (int d = 0; d < DIM; ++d) {
                    const T lam = PDE::max_eig(P.pde, qs, d);
                    bad |= !(lam >= T(0));
                    lmax[d] = lam > lmax[d] ? lam : lmax[d];
                }
            }
            if (g + 1 < ngrp) usync();  // buffer b, the face fluxes and the reference differences are reused
        }
        if constexpr (C::WM) {
            if (S.ctl != acc_ctl) {  // warp-uniform: a new solve
                flush();
                acc_ctl = S.ctl;
            }
#pragma unroll
            for (int d = 0; d < DIM; ++d) acc_l[d] = lmax[d] > acc_l[d] ? lmax[d] : acc_l[d];
            acc_bad |= bad;
        } else {
#pragma unroll
            for (int d = 0; d < DIM; ++d) {
                T x = lmax[d];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const T y = __shfl_xor_sync(0xffffffffu, x, o);
                    x = y > x ? y : x;
                }
                lmax[d] = x;
            }
            const unsigned anybad = __any_sync(0xffffffffu, bad);
            const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
            // the CTA's maxima in the compute type (on the FP32 path no FP64
            // instruction: one costs the whole warp's FP64 issue slot however
            // few lanes it has); widened once for the atomic
            T *redT = reinterpret_cast<T *>(red);
            int *redB = reinterpret_cast<int *>(red + 64);
            if (lane == 0) {
#pragma unroll
                for (int d = 0; d < DIM; ++d) redT[warp * 4 + d] = lmax[d];
                redB[warp] = anybad ? 1 : 0;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                const int nw = blockDim.x >> 5;
                int b = 0;
                for (int d = 0; d < DIM; ++d) {
                    T x = T(0);
                    for (int w = 0; w < nw; ++w) x = tmax(x, redT[w * 4 + d]);
                    atomicMax(&S.ctl->lam_acc[d], (unsigned long long)__double_as_longlong(double(x)));
                }
                for (int w = 0; w < nw; ++w) b |= redB[w];
                if (b) atomicOr(&S.ctl->flags, FLAG_NONFINITE);
            }
        }
        usync();  // shared buffers are reused by the next tile
    }
    if constexpr (C::WM) flush();
}

// the subcell limiter's sizes (limiter.cuh)
template <class PDE, int DIM, int N>
struct LimCfg;

// Wave-speed maxima of the current state of solve 0 of the launch (the CFL
// input of the first step after an upload, and after a limited step that
// changed the state): grid-stride over all nodes, one atomic per warp.
template <class PDE, int DIM, int N, typename T>
__global__ void __launch_bounds__(256) k_cfl(const KParams P)
{
    using G = Geom<PDE, DIM, N>;
    constexpr int M = G::M;
    const SolveDesc &S = P.solves[0];
    // after a limited step that troubled no element the state is the
    // corrector's candidate: its maxima stand
    if (P.lim_pass && S.ctl->lim_count == 0u) return;
    // kept subcell data (Sec. 2.3): the elements lim_flags marks are limited
    // ones, whose wave speeds are those of their subcell averages (lim_subn,
    // listed in lim_list), not of the nodes of the reconstructed polynomial
    const bool kept = S.lim_sub && S.ctl->lim_kept_ok != 0;
    const long long total = S.E * G::NS;
    double lmax[DIM];
#pragma unroll
    for (int d = 0; d < DIM; ++d) lmax[d] = 0.0;
    bool bad = false;
    auto take = [&](const double *a) {
        T q[M];
#pragma unroll
        for (int v = 0; v < M; ++v) {
            const double x = a[v];
            bad |= dbl_nonfinite(x);
            q[v] = narrow<T>(x);
        }
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            const double lam = double(PDE::max_eig(P.pde, q, d));
            bad |= !(lam >= 0.0);
            lmax[d] = fmax(lmax[d], lam);
        }
    };
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        if (kept && S.lim_flags[i / G::NS]) {
#pragma unroll
            for (int v = 0; v < M; ++v) bad |= dbl_nonfinite(S.u[i * M + v]);
            continue;
        }
        take(S.u + i * M);
    }
    if constexpr (LimCfg<PDE, DIM, N>::OK) {
        if (kept) {
            constexpr int NSUB = LimCfg<PDE, DIM, N>::NSUB;
            const long long nk = (long long)min(S.ctl->lim_count, (unsigned)S.E) * NSUB;
            for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < nk;
                 j += (long long)gridDim.x * blockDim.x) {
                const long long e = S.lim_list[j / NSUB];
                take(S.lim_subn + (e * NSUB + j % NSUB) * M);
            }
        }
    }
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        double x = lmax[d];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(0xffffffffu, x, o));
        if ((threadIdx.x & 31) == 0) atomicMax(&S.ctl->lam_acc[d], (unsigned long long)__double_as_longlong(x));
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&S.ctl->flags, FLAG_NONFINITE);
}

#include "limiter.cuh"

// The limiter's kernels of one (PDE, d, N); K: 0 minmax, 1 detect, 2 fv,
// 3 couple, 4 / 5 the FP32 path's minmax / detect, 6 the subcell-data
// upload, 7 / 8 the minmax kernels of solves that keep subcell data.  Detection and the subcell scheme work on the FP64 state in
// both precisions and are referenced by the FP64 instance only (so that
// each is compiled once; an FP32-path handle takes them from there); the
// coupling replaces the face fluxes of the step's own precision.
using KernelFn = void (*)(KParams);
template <class PDE, int DIM, int N, typename T, int K>
constexpr KernelFn lim_kernel()
{
    if constexpr (LimCfg<PDE, DIM, N>::OK && sizeof(T) == 8) {
        if constexpr (K == 0) return &k_lim_minmax<PDE, DIM, N, false>;
        else if constexpr (K == 1) return &k_lim_detect<PDE, DIM, N>;
        else if constexpr (K == 2) return &k_lim_fv<PDE, DIM, N>;
        else if constexpr (K == 4) return &k_lim_minmax32<PDE, DIM, N, false>;
        else if constexpr (K == 7) return &k_lim_minmax<PDE, DIM, N, true>;
        else if constexpr (K == 8) return &k_lim_minmax32<PDE, DIM, N, true>;
        else if constexpr (K == 5) return &k_lim_detect32<PDE, DIM, N>;
        else if constexpr (K == 6) return &k_lim_subcell_init<PDE, DIM, N>;
        else return &k_lim_couple<PDE, DIM, N, T>;
    } else if constexpr (LimCfg<PDE, DIM, N>::OK && K == 3) {
        return &k_lim_couple<PDE, DIM, N, T>;
    } else {
        return nullptr;
    }
}

template <class PDE, int DIM, int N, typename T>
struct KS {
    static const KernelSet value;
};

// Predictor shapes: 0-2 k_predictor with CTAs of the default, half and
// double size; 3-4 the plane-owning k_predictor_xt (about 128 and 256
// threads) where it applies (2D FP32, small planes), else shapes 0 and 2.
template <class PDE, int DIM, int N, typename T, int TS, bool EX = false>
constexpr TileShape pred_shape()
{
    if constexpr (TS >= 7) {
        if constexpr (PredCfg<PDE, DIM, N, T, TS>::QX) {
            using C = PredCfg<PDE, DIM, N, T, TS>;  // shapes 0 / 1 exchanging the state (FP32, conservative)
            return TileShape{&k_predictor<PDE, DIM, N, T, TS, EX>, C::THREADS, C::EPB, C::BYTES};
        } else {
            return pred_shape<PDE, DIM, N, T, TS - 7, EX>();  // repeats of shapes 0 and 1
        }
    } else if constexpr (TS >= 5) {
        if constexpr (PredCfg<PDE, DIM, N, T, TS>::TC) {
            using C = PredCfg<PDE, DIM, N, T, TS>;  // shapes 0 / 1 with tensor-core contractions (FP32)
            return TileShape{&k_predictor<PDE, DIM, N, T, TS, EX>, C::THREADS, C::EPB, C::BYTES};
        } else {
            return pred_shape<PDE, DIM, N, T, TS - 5, EX>();  // FP64: repeats of shapes 0 and 1
        }
    } else if constexpr (TS >= 3) {
        if constexpr (DIM == 2 && sizeof(T) == 4 && use_xt<PDE, N>()) {
            using C = PredXtCfg<PDE, N, TS == 3 ? 0 : 2>;
            return TileShape{&k_predictor_xt<PDE, N, TS == 3 ? 0 : 2, EX>, C::THREADS, C::EPB, C::BYTES};
        } else {
            return pred_shape<PDE, DIM, N, T, TS == 3 ? 0 : 2, EX>();
        }
    } else {
        using C = PredCfg<PDE, DIM, N, T, TS>;
        return TileShape{&k_predictor<PDE, DIM, N, T, TS, EX>, C::THREADS, C::EPB, C::BYTES};
    }
}

template <class PDE, int DIM, int N, typename T, int TS>
constexpr TileShape corr_shape()
{
    using C = CorrCfg<PDE, DIM, N, T, TS>;
    return TileShape{&k_corrector<PDE, DIM, N, T, TS>, C::THREADS, C::EPB_TILE, C::CTA_BYTES};
}

template <class PDE, int DIM, int N, typename T>
const KernelSet KS<PDE, DIM, N, T>::value = {
    pred_shape<PDE, DIM, N, T, 0>().kernel, pred_shape<PDE, DIM, N, T, 0>().threads,
    pred_shape<PDE, DIM, N, T, 0>().epb, pred_shape<PDE, DIM, N, T, 0>().smem,
    &k_corrector<PDE, DIM, N, T, 0>, CorrCfg<PDE, DIM, N, T>::THREADS, CorrCfg<PDE, DIM, N, T>::EPB,
    CorrCfg<PDE, DIM, N, T>::BYTES,
    &k_cfl<PDE, DIM, N, T>,
    Geom<PDE, DIM, N>::M, Geom<PDE, DIM, N>::RS, (int)sizeof(T), PDE::FLUX_FLOPS, PDE::EIG_FLOPS,
    PredCfg<PDE, DIM, N, T>::DELTA ? PredCfg<PDE, DIM, N, T>::RF : 0, PDE::NCP ? 1 : 0, PredCfg<PDE, DIM, N, T>::MX,
    lim_kernel<PDE, DIM, N, T, 0>(), lim_kernel<PDE, DIM, N, T, 1>(), lim_kernel<PDE, DIM, N, T, 2>(),
    lim_kernel<PDE, DIM, N, T, 3>(), LimCfg<PDE, DIM, N>::BYTES, LimWarp<LimCfg<PDE, DIM, N>>::BYTES,
    lim_kernel<PDE, DIM, N, T, 4>(), lim_kernel<PDE, DIM, N, T, 5>(), LimWarp32<LimCfg<PDE, DIM, N>>::BYTES,
    lim_kernel<PDE, DIM, N, T, 6>(), lim_kernel<PDE, DIM, N, T, 7>(), lim_kernel<PDE, DIM, N, T, 8>(),
    {pred_shape<PDE, DIM, N, T, 0>(), pred_shape<PDE, DIM, N, T, 1>(), pred_shape<PDE, DIM, N, T, 2>(),
     pred_shape<PDE, DIM, N, T, 3>(), pred_shape<PDE, DIM, N, T, 4>(), pred_shape<PDE, DIM, N, T, 5>(),
     pred_shape<PDE, DIM, N, T, 6>(), pred_shape<PDE, DIM, N, T, 7>(), pred_shape<PDE, DIM, N, T, 8>()},
    {pred_shape<PDE, DIM, N, T, 0, true>(), pred_shape<PDE, DIM, N, T, 1, true>(),
     pred_shape<PDE, DIM, N, T, 2, true>(), pred_shape<PDE, DIM, N, T, 3, true>(),
     pred_shape<PDE, DIM, N, T, 4, true>(), pred_shape<PDE, DIM, N, T, 5, true>(),
     pred_shape<PDE, DIM, N, T, 6, true>(), pred_shape<PDE, DIM, N, T, 7, true>(),
     pred_shape<PDE, DIM, N, T, 8, true>()},
    {corr_shape<PDE, DIM, N, T, 0>(), corr_shape<PDE, DIM, N, T, 1>(), corr_shape<PDE, DIM, N, T, 2>(),
     corr_shape<PDE, DIM, N, T, 3>(), corr_shape<PDE, DIM, N, T, 4>(), corr_shape<PDE, DIM, N, T, 5>()},
    0, 0};

}  // namespace aderdg
