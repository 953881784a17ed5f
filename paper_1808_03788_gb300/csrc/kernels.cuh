// Element-batch kernels of the ADER-DG step, templated on the PDE, the
// dimension, the degree and the compute type T (double: FP64 path; float:
// mixed path whose state update stays in double).
//
//  k_predictor  space-time predictor (Sec. 2.2, eq. pde.st2) by Picard
//               iteration, time averages, volume integral, face traces
//  k_corrector  Rusanov fluxes on the time-averaged traces (eq. pc.scheme
//               with B = 0, eq. rusanov), surface lift and element update
//               (eq. pde.nc.gw2), wave-speed maxima for the next CFL step
//
// One CTA holds EPB elements; each element is worked on by a group of
// threads, one per space-time node (predictor) or spatial node (corrector).
// The element's working set lives in shared memory and registers, so u^n is
// read once and the space-time DOFs never touch HBM (the cache-blocking
// property of Sec. 2.2 mapped onto an SM).
#pragma once

#include "common.cuh"

namespace aderdg {

template <typename T>
__device__ __forceinline__ T tmax(T a, T b) { return a > b ? a : b; }

// shared-memory footprint (bytes) of the predictor, shared part + per group
template <class PDE, int DIM, int N, typename T>
struct PredSmem {
    using G = Geom<PDE, DIM, N>;
    static constexpr int SHARED = round_up(3 * G::n * G::n + 3 * G::n, 2);
    // work buffer: space-time values, later the per-face traces
    static constexpr int BUFN = G::NST > G::NREC ? G::NST : G::NREC;
    static constexpr int GROUP = BUFN * G::M + G::NS * G::M * (2 + DIM);
    static constexpr size_t BYTES = sizeof(T) * (size_t)(SHARED + G::P_EPB * GROUP);
};

template <class PDE, int DIM, int N, typename T>
__global__ void __launch_bounds__(Geom<PDE, DIM, N>::P_THREADS)
k_predictor(const KParams P)
{
    using G = Geom<PDE, DIM, N>;
    using S = PredSmem<PDE, DIM, N, T>;
    constexpr int n = G::n, M = G::M, NS = G::NS, NST = G::NST, NF = G::NF;
    constexpr int TPE = G::P_TPE, EPB = G::P_EPB, RS = G::RS;

    const double dt = P.use_ctl_dt ? P.ctl->dt : P.dt_arg;
    if (!(dt > 0.0)) return;  // uniform over the grid: no step in flight

    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sD = reinterpret_cast<T *>(smem_raw);
    T *sA = sD + n * n;     // dt * iK1 W
    T *sK = sA + n * n;     // Kw
    T *sF0 = sK + n * n;
    T *sF1 = sF0 + n;
    T *sw = sF1 + n;
    const int g = threadIdx.x / TPE;
    const int l = threadIdx.x - g * TPE;
    T *buf = reinterpret_cast<T *>(smem_raw) + S::SHARED + g * S::GROUP;  // BUFN*M
    T *qbar = buf + S::BUFN * M;      // NS*M
    T *Fbar = qbar + NS * M;          // DIM*NS*M
    T *us = Fbar + DIM * NS * M;      // NS*M

    for (int i = threadIdx.x; i < n * n; i += blockDim.x) {
        sD[i] = T(P.b.D[i]);
        sA[i] = T(dt * P.b.iK1W[i]);
        sK[i] = T(P.b.Kw[i]);
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        sF0[i] = T(P.b.F0[i]);
        sF1[i] = T(P.b.F1[i]);
        sw[i] = T(P.b.w[i]);
    }

    const long long e = (long long)blockIdx.x * EPB + g;
    const bool valid = e < P.E;
    const long long ec = valid ? e : P.E - 1;  // tail groups recompute the last element
    const double *ue = P.u + ec * (NS * M);
    for (int i = l; i < NS * M; i += TPE) us[i] = T(ue[i]);
    __syncthreads();

    const int node = l;
    const bool act = node < NST;
    const int t = act ? node / NS : 0;
    const int s = act ? node - t * NS : 0;
    int sd[DIM];
    {
        int r = s;
#pragma unroll
        for (int d = 0; d < DIM; ++d) { sd[d] = r % n; r /= n; }
    }
    T u0[M], q[M];
#pragma unroll
    for (int v = 0; v < M; ++v) { u0[v] = us[s * M + v]; q[v] = u0[v]; }

    // ---- Picard iterations of eq. pde.st2 --------------------------------
    for (int it = 0; it < P.picard; ++it) {
        T F[DIM][M];
        PDE::flux(P.pde, q, F);
        T R[M];
#pragma unroll
        for (int v = 0; v < M; ++v) R[v] = T(0);
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            if (act) {
#pragma unroll
                for (int v = 0; v < M; ++v) buf[node * M + v] = F[d][v];
            }
            __syncthreads();
            if (act) {
                const int stride = ipow(n, d);
                const int base = node - sd[d] * stride;
                const T *Drow = sD + sd[d] * n;
                const T idx = T(P.inv_dx[d]);
#pragma unroll
                for (int v = 0; v < M; ++v) {
                    T acc = T(0);
#pragma unroll
                    for (int j = 0; j < n; ++j) acc += Drow[j] * buf[(base + j * stride) * M + v];
                    R[v] -= idx * acc;
                }
            }
            __syncthreads();
        }
        if (act) {
#pragma unroll
            for (int v = 0; v < M; ++v) buf[node * M + v] = R[v];
        }
        __syncthreads();
        if (act) {
            const T *Arow = sA + t * n;
#pragma unroll
            for (int v = 0; v < M; ++v) {
                T acc = T(0);
#pragma unroll
                for (int tp = 0; tp < n; ++tp) acc += Arow[tp] * buf[(tp * NS + s) * M + v];
                q[v] = u0[v] + acc;
            }
        }
        __syncthreads();
    }

    // ---- time averages qbar, Fbar_d --------------------------------------
    T F[DIM][M];
    PDE::flux(P.pde, q, F);
    if (act) {
#pragma unroll
        for (int v = 0; v < M; ++v) buf[node * M + v] = q[v];
    }
    __syncthreads();
    for (int i = l; i < NS * M; i += TPE) {
        T acc = T(0);
#pragma unroll
        for (int tt = 0; tt < n; ++tt) acc += sw[tt] * buf[tt * NS * M + i];
        qbar[i] = acc;
    }
    __syncthreads();
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        if (act) {
#pragma unroll
            for (int v = 0; v < M; ++v) buf[node * M + v] = F[d][v];
        }
        __syncthreads();
        for (int i = l; i < NS * M; i += TPE) {
            T acc = T(0);
#pragma unroll
            for (int tt = 0; tt < n; ++tt) acc += sw[tt] * buf[tt * NS * M + i];
            Fbar[d * NS * M + i] = acc;
        }
        __syncthreads();
    }

    // ---- volume term V = sum_d (1/dx_d) Kw_d Fbar_d ------------------------
    T *Vout = reinterpret_cast<T *>(P.V) + ec * (NS * M);
    for (int i = l; i < NS * M; i += TPE) {
        const int si = i / M, v = i - si * M;
        T acc = T(0);
        int r = si;
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            const int k = r % n;
            r /= n;
            const int stride = ipow(n, d);
            const int base = si - k * stride;
            const T *Krow = sK + k * n;
            T a = T(0);
#pragma unroll
            for (int j = 0; j < n; ++j) a += Krow[j] * Fbar[(d * NS + base + j * stride) * M + v];
            acc += T(P.inv_dx[d]) * a;
        }
        if (valid) Vout[i] = acc;
    }

    // ---- face traces of the time averages ----------------------------------
    T *trE = reinterpret_cast<T *>(P.tr) + ec * (G::NREC * RS);
    for (int i = l; i < G::NREC * M; i += TPE) {
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
            aq += phi[j] * qbar[(s0 + j * pd) * M + v];
            af += phi[j] * Fbar[(d * NS + s0 + j * pd) * M + v];
        }
        buf[rec * M + v] = aq;  // for the wave speed below
        if (valid) {
            trE[rec * RS + v] = aq;
            trE[rec * RS + M + v] = af;
        }
    }
    __syncthreads();
    for (int rec = l; rec < G::NREC; rec += TPE) {
        const int d = rec / (2 * NF);
        const T lam = PDE::max_eig(P.pde, buf + rec * M, d);
        if (valid) {
            trE[rec * RS + 2 * M] = lam;
            trE[rec * RS + 2 * M + 1] = T(0);
        }
    }
}

template <class PDE, int DIM, int N, typename T>
struct CorrSmem {
    using G = Geom<PDE, DIM, N>;
    static constexpr int SHARED = 3 * NMAX;  // F0, F1, 1/w (double)
    static constexpr int GROUP = G::NREC * G::M + G::NS * G::M;  // F*, u^{n+1}
    static constexpr size_t BYTES = sizeof(double) * SHARED + sizeof(T) * (size_t)G::C_EPB * G::NREC * G::M
                                    + sizeof(double) * (size_t)G::C_EPB * G::NS * G::M + 64 * sizeof(double);
};

__device__ __forceinline__ long long neighbour(long long e, const int *cells, int d, int off)
{
    long long idx[3] = {0, 0, 0}, r = e;
    idx[0] = r % cells[0]; r /= cells[0];
    idx[1] = r % cells[1]; r /= cells[1];
    idx[2] = r;
    long long c = idx[d] + off;
    if (c < 0) c += cells[d];
    if (c >= cells[d]) c -= cells[d];
    idx[d] = c;
    return idx[0] + (long long)cells[0] * (idx[1] + (long long)cells[1] * idx[2]);
}

template <class PDE, int DIM, int N, typename T>
__global__ void __launch_bounds__(Geom<PDE, DIM, N>::C_THREADS)
k_corrector(const KParams P)
{
    using G = Geom<PDE, DIM, N>;
    constexpr int n = G::n, M = G::M, NS = G::NS, NF = G::NF, RS = G::RS;
    constexpr int TPE = G::C_TPE, EPB = G::C_EPB, NREC = G::NREC;

    const double dt = P.use_ctl_dt ? P.ctl->dt : P.dt_arg;
    if (!(dt > 0.0)) return;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    double *sF0 = reinterpret_cast<double *>(smem_raw);
    double *sF1 = sF0 + NMAX;
    double *sIw = sF1 + NMAX;
    double *red = sIw + NMAX;  // 64 doubles for the block reduction
    const int g = threadIdx.x / TPE;
    const int l = threadIdx.x - g * TPE;
    double *un = red + 64 + g * (NS * M);
    T *Fs = reinterpret_cast<T *>(red + 64 + EPB * NS * M) + g * (NREC * M);

    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        sF0[i] = P.b.F0[i];
        sF1[i] = P.b.F1[i];
        sIw[i] = P.b.inv_w[i];
    }
    const long long e = (long long)blockIdx.x * EPB + g;
    const bool valid = e < P.E;
    const long long ec = valid ? e : P.E - 1;
    const T *tr = reinterpret_cast<const T *>(P.tr);

    // ---- Rusanov flux on every face node of this element -------------------
    for (int i = l; i < NREC * M; i += TPE) {
        const int rec = i / M, v = i - rec * M;
        const int d = rec / (2 * NF);
        const int side = (rec / NF) & 1;
        const int p = rec - (rec / NF) * NF;
        const long long en = neighbour(ec, P.cells, d, side ? 1 : -1);
        const T *own = tr + (ec * NREC + rec) * RS;
        const T *nb = tr + (en * NREC + (rec + (side ? -NF : NF))) * RS;
        const T *L = side ? own : nb;
        const T *R = side ? nb : own;
        const T smax = tmax(L[2 * M], R[2 * M]);
        Fs[rec * M + v] = T(0.5) * (L[M + v] + R[M + v]) - T(0.5) * smax * (R[v] - L[v]);
        (void)p;
    }
    __syncthreads();

    // ---- surface lift and update u^{n+1} = u^n + dt (V - surface) ----------
    const double *ue = P.u + ec * (NS * M);
    const T *Ve = reinterpret_cast<const T *>(P.V) + ec * (NS * M);
    double *uo = P.u_out + ec * (NS * M);
    for (int i = l; i < NS * M; i += TPE) {
        const int si = i / M, v = i - si * M;
        T surf = T(0);
        int r = si;
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            const int k = r % n;
            r /= n;
            const int pd = ipow(n, d);
            const int p = (si % pd) + (si / (pd * n)) * pd;
            const T fp = Fs[((d * 2 + 1) * NF + p) * M + v];
            const T fm = Fs[((d * 2 + 0) * NF + p) * M + v];
            surf += T(P.inv_dx[d] * sIw[k]) * (T(sF1[k]) * fp - T(sF0[k]) * fm);
        }
        const double unew = ue[i] + dt * double(Ve[i] - surf);
        un[i] = unew;
        if (valid) uo[i] = unew;
    }
    __syncthreads();

    // ---- wave-speed maxima of u^{n+1} and non-finite check -----------------
    double lmax[DIM];
#pragma unroll
    for (int d = 0; d < DIM; ++d) lmax[d] = 0.0;
    bool bad = false;
    if (valid) {
        for (int si = l; si < NS; si += TPE) {
            T qs[M];
#pragma unroll
            for (int v = 0; v < M; ++v) {
                const double x = un[si * M + v];
                bad |= !isfinite(x);
                qs[v] = T(x);
            }
#pragma unroll
            for (int d = 0; d < DIM; ++d) {
                const double lam = double(PDE::max_eig(P.pde, qs, d));
                bad |= !(lam >= 0.0);
                lmax[d] = fmax(lmax[d], lam);
            }
        }
    }
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        double x = lmax[d];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(0xffffffffu, x, o));
        lmax[d] = x;
    }
    const unsigned anybad = __any_sync(0xffffffffu, bad);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();  // 'red' is free: everyone is past the update loop
    if (lane == 0) {
#pragma unroll
        for (int d = 0; d < DIM; ++d) red[warp * 4 + d] = lmax[d];
        red[warp * 4 + 3] = anybad ? 1.0 : 0.0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nw = blockDim.x >> 5;
        double b = 0.0;
        for (int d = 0; d < DIM; ++d) {
            double x = 0.0;
            for (int w = 0; w < nw; ++w) x = fmax(x, red[w * 4 + d]);
            atomicMax(&P.ctl->lam_acc[d], (unsigned long long)__double_as_longlong(x));
        }
        for (int w = 0; w < nw; ++w) b = fmax(b, red[w * 4 + 3]);
        if (b > 0.0) atomicOr(&P.ctl->flags, FLAG_NONFINITE);
    }
}

// Wave-speed maxima of the current state (the CFL input of the first step
// after a state upload): grid-stride over all nodes, one atomic per warp.
template <class PDE, int DIM, int N, typename T>
__global__ void __launch_bounds__(256) k_cfl(const KParams P)
{
    using G = Geom<PDE, DIM, N>;
    constexpr int M = G::M;
    const long long total = P.E * G::NS;
    double lmax[DIM];
#pragma unroll
    for (int d = 0; d < DIM; ++d) lmax[d] = 0.0;
    bool bad = false;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        T q[M];
#pragma unroll
        for (int v = 0; v < M; ++v) {
            const double x = P.u[i * M + v];
            bad |= !isfinite(x);
            q[v] = T(x);
        }
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            const double lam = double(PDE::max_eig(P.pde, q, d));
            bad |= !(lam >= 0.0);
            lmax[d] = fmax(lmax[d], lam);
        }
    }
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        double x = lmax[d];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(0xffffffffu, x, o));
        if ((threadIdx.x & 31) == 0) atomicMax(&P.ctl->lam_acc[d], (unsigned long long)__double_as_longlong(x));
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&P.ctl->flags, FLAG_NONFINITE);
}

template <class PDE, int DIM, int N, typename T>
struct KS {
    using G = Geom<PDE, DIM, N>;
    static const KernelSet value;
};

template <class PDE, int DIM, int N, typename T>
const KernelSet KS<PDE, DIM, N, T>::value = {
    &k_predictor<PDE, DIM, N, T>, G::P_THREADS, G::P_EPB, PredSmem<PDE, DIM, N, T>::BYTES,
    &k_corrector<PDE, DIM, N, T>, G::C_THREADS, G::C_EPB, CorrSmem<PDE, DIM, N, T>::BYTES,
    &k_cfl<PDE, DIM, N, T>,
    G::M, G::RS, (int)sizeof(T), PDE::FLUX_FLOPS, PDE::EIG_FLOPS};

}  // namespace aderdg
