// Space-time predictor of the 2D FP32 path with (x, t)-plane ownership.
//
// Thread (element, y) owns the n x n space-time nodes (t, x) at its y, all
// m variables, in registers.  The flux, the x-derivative, the time solve
// q = u + dt iK1W R and the time averages are register-local; only the
// y-derivative passes through shared memory: F_y is written, -Dhat F_y is
// taken along y in place (thread y takes the pencils (t, x = y)), and the
// result is read back -- 4 NST m values per element and iteration, half of
// what the time-pencil layout of k_predictor moves (2 d NST m through
// shared memory and back).  The arithmetic per value is the same as
// k_predictor's (eq. pde.st2, perturbation form about the element's
// reference node; initial guesses of Sec. 2.2).
// Included by kernels.cuh inside namespace aderdg.
#pragma once

// Used where the plane fits the registers: n^2 m <= 100 floats (2D Euler
// N <= 4, 2D advection N <= 9); larger orders and the purely
// non-conservative systems keep k_predictor.
template <class PDE, int N>
constexpr bool use_xt() { return !PDE::NCP && (N + 1) * (N + 1) * PDE::M <= 100; }

template <class PDE, int N, int TS>
struct PredXtCfg {
    using G = Geom<PDE, 2, N>;
    static constexpr int n = G::n, M = G::M, NS = G::NS, NST = G::NST, NF = G::NF, NREC = G::NREC, RS = G::RS;
    // shapes 0, 1, 2: about 128, 64, 256 threads
    static constexpr int TARGET = TS == 1 ? 64 : (TS == 2 ? 256 : 128);
    static constexpr int EPB = cmax(1, TARGET / n);
    static constexpr int THREADS = round_up(EPB * n, 32);
    // shape 0 (about 128 threads): 3 CTAs per SM (168 registers; large planes
    // spill a little); shape 2 (about 256 threads): one CTA, up to 255 registers
    static constexpr int MINB = TS == 2 ? 1 : cmax(1, (3 * 128) / THREADS);
    // per element: the F_y / R_y field [t][y][x][v]; its size is padded to
    // 16 mod 128 bytes so that neighbouring elements start on other banks
    static constexpr int ELEM = round_up(NST * M, 32) + 4;
    // per CTA: dt / dx_0, then Kw and the face values (rows indexed by y),
    // the extrapolation weights [t][k]
    static constexpr int HEAD = round_up(1 + n * n + 2 * n + n * n, 4);
    static constexpr size_t BYTES = sizeof(float) * ((size_t)HEAD + (size_t)EPB * ELEM);
    static constexpr int SREF = NS / 2;
    static constexpr int RF = M;
    static constexpr bool DELTA = true;
};

// -Dhat along y on the pencil (t, x) of the field f[t][y][x][v], in place,
// all variables; same FMA order as contract_pencil.
template <int n, int M>
__device__ __forceinline__ void xt_contract_y(float *f, int t, int x, const float *Dm)
{
    using IO = NodeIO<float, M>;
    constexpr int NS = n * n;
    float *base = f + (t * NS + x) * M;
    float a[n][M];
#pragma unroll
    for (int j = 0; j < n; ++j) IO::load(base + j * n * M, a[j]);
#pragma unroll
    for (int i = 0; i < n; ++i) {
        float r[M];
#pragma unroll
        for (int v = 0; v < M; ++v) {
            float acc = Dm[i * n] * a[0][v];
#pragma unroll
            for (int j = 1; j < n; ++j) acc += Dm[i * n + j] * a[j][v];
            r[v] = acc;
        }
        IO::store(base + i * n * M, r);
    }
}

// -Dhat along x of a row F[x][v] held in registers: R[i] = sum_j Dm[i][j] F[j].
template <int n, int M>
__device__ __forceinline__ void xt_contract_x(const float (*F)[M], float (*R)[M], const float *Dm)
{
#pragma unroll
    for (int i = 0; i < n; ++i)
#pragma unroll
        for (int v = 0; v < M; ++v) {
            float acc = Dm[i * n] * F[0][v];
#pragma unroll
            for (int j = 1; j < n; ++j) acc += Dm[i * n + j] * F[j][v];
            R[i][v] = acc;
        }
}

template <class PDE, int N, int TS, bool EX>
__global__ void __launch_bounds__(PredXtCfg<PDE, N, TS>::THREADS, PredXtCfg<PDE, N, TS>::MINB)
k_predictor_xt(const KParams P)
{
    using C = PredXtCfg<PDE, N, TS>;
    constexpr int n = C::n, M = C::M, NS = C::NS, NF = C::NF, NREC = C::NREC, RS = C::RS, EPB = C::EPB;
    using IO = NodeIO<float, M>;
    const Ops<float> &O = P.of;
    const float *Dm = O.Dm[0];

    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *sHead = reinterpret_cast<float *>(smem_raw);
    float *sDt = sHead;               // dt / dx_0 of the current tile
    float *sKw = sHead + 1;           // Kw [k][j]
    float *sF0 = sKw + n * n;         // face values at xi = 0 and 1
    float *sF1 = sF0 + n;
    float *sW = sF1 + n;              // extrapolation weights of the tile
    const int tid = threadIdx.x;
    const bool act = tid < EPB * n;
    const int g = act ? tid / n : 0;
    const int y = act ? tid - g * n : 0;
    float *eb = sHead + C::HEAD + g * C::ELEM;  // F_y / R_y [t][y][x][v]; later qbar | Fbar_y [y][x][v]

    for (int i = tid; i < n * n; i += blockDim.x) sKw[i] = O.Kv[0][i];
    for (int i = tid; i < n; i += blockDim.x) {
        sF0[i] = O.F0[i];
        sF1[i] = O.F1[i];
    }
    __syncthreads();

    for (long long tile = blockIdx.x; tile < P.ntiles; tile += gridDim.x) {
        const int si = find_solve(P.solves, P.nsolves, tile, 0);
        const SolveDesc &S = P.solves[si];
        const double dt = solve_dt(P, S);
        if (!(dt > 0.0)) continue;  // uniform over the CTA
        if (tid == 0) sDt[0] = float(dt * S.inv_dx[0]);
        const float ratio1 = S.ratio_f[1];  // dx_0 / dx_1
        const float idx0 = S.inv_dx_f[0], idx1 = S.inv_dx_f[1];
        const float dx0 = float(1.0 / S.inv_dx[0]);

        const long long e = (tile - S.tile0_p) * EPB + g;
        const bool valid = act && e < S.E;
        const long long el = e < S.E ? e : S.E - 1;
        const long long ec = S.elist ? (long long)S.elist[el] : el;  // a listed subset of a block, or all

        // reference state (node SREF) and the perturbations u - u_ref of this
        // thread's row of nodes (x, y)
        typename PDE::template Ref<float> ref;
        double uref[M];
#pragma unroll
        for (int v = 0; v < M; ++v) uref[v] = S.u[(ec * NS + C::SREF) * M + v];
        {
            float urf[M];
#pragma unroll
            for (int v = 0; v < M; ++v) urf[v] = dbl_to_flt_rn(uref[v]);
            PDE::make_ref(P.pde, urf, ref);
        }
        // dx_0 S(ref + w) added to R (linear algebraic source, Sec. 2.1)
        auto add_src = [&](const float *w, float *R) {
            if constexpr (PDE::HAS_SRC) {
                float qa[M], Sq[M];
#pragma unroll
                for (int v = 0; v < M; ++v) qa[v] = w[v] + ref.q[v];
                PDE::source(P.pde, qa, Sq);
#pragma unroll
                for (int v = 0; v < M; ++v) R[v] += dx0 * Sq[v];
            }
        };
        float u[n][M];
#pragma unroll
        for (int x = 0; x < n; ++x)
#pragma unroll
            for (int v = 0; v < M; ++v) u[x][v] = dbl_to_flt_rn(S.u[(ec * NS + y * n + x) * M + v] - uref[v]);
        __syncthreads();  // sDt, and eb free (previous tile)
        const float dtT = sDt[0];

        // R(w) = dx_0 L(w) of the time-constant row w[x] (Sec. 2.2): F_x
        // derivative in registers, F_y through the t = 0 slice of eb
        auto spatial_R = [&](const float (*w)[M], float (*R)[M]) {
            float Fx[n][M];
#pragma unroll
            for (int x = 0; x < n; ++x) {
                float F[2][M];
                PDE::flux_delta(P.pde, ref, w[x], F);
#pragma unroll
                for (int v = 0; v < M; ++v) Fx[x][v] = F[0][v];
                if (act) IO::store(eb + (y * n + x) * M, F[1]);
            }
            xt_contract_x<n, M>(Fx, R, Dm);
            __syncthreads();
            if (act) xt_contract_y<n, M>(eb, 0, y, Dm);
            __syncthreads();
#pragma unroll
            for (int x = 0; x < n; ++x) {
                float r[M];
                IO::load(eb + (y * n + x) * M, r);
#pragma unroll
                for (int v = 0; v < M; ++v) R[x][v] += ratio1 * r[v];
                add_src(w[x], R[x]);
            }
            __syncthreads();
        };

        float A[n][n][M];  // [t][x][v]: q, then F_x and R in place
        int it0;
        int P_it = S.picard;
        bool extrap = false;
        if constexpr (EX) extrap = S.guess == 3 && P.use_ctl_dt && S.ctl->dt_prev > 0.0;
        if (extrap) {
            // extrapolation of the previous step's predictor (Sec. 2.2)
            if (tid == 0) extrap_weights<float, n>(O, float(dt / S.ctl->dt_prev), sW);
            __syncthreads();
            const float *qp = reinterpret_cast<const float *>(S.qprev) + ec * (n * NS * M);
#pragma unroll
            for (int t = 0; t < n; ++t)
#pragma unroll
                for (int x = 0; x < n; ++x)
#pragma unroll
                    for (int v = 0; v < M; ++v) A[t][x][v] = u[x][v];
#pragma unroll 1
            for (int k = 0; k < n; ++k) {  // one previous time level at a time
#pragma unroll
                for (int x = 0; x < n; ++x) {
                    float qk[M];
                    IO::load(qp + (k * NS + y * n + x) * M, qk);
#pragma unroll
                    for (int t = 0; t < n; ++t) {
                        const float wk = sW[t * n + k];
#pragma unroll
                        for (int v = 0; v < M; ++v) A[t][x][v] += wk * qk[v];
                    }
                }
            }
            it0 = 0;
        } else {
            float R1[n][M];
            spatial_R(u, R1);
            if (S.guess == 3) P_it = S.picard_first;  // no previous predictor: the third-order guess
            if (S.guess == 2 || S.guess == 3) {
                float w[n][M], R2[n][M];
#pragma unroll
                for (int x = 0; x < n; ++x)
#pragma unroll
                    for (int v = 0; v < M; ++v) w[x][v] = u[x][v] + dtT * R1[x][v];
                spatial_R(w, R2);
#pragma unroll
                for (int t = 0; t < n; ++t)
#pragma unroll
                    for (int x = 0; x < n; ++x)
#pragma unroll
                        for (int v = 0; v < M; ++v)
                            A[t][x][v] = u[x][v] + dtT * (O.xi[t] * R1[x][v] + O.hxi2[t] * (R2[x][v] - R1[x][v]));
                it0 = 0;
            } else if (S.guess == 1) {
#pragma unroll
                for (int t = 0; t < n; ++t)
#pragma unroll
                    for (int x = 0; x < n; ++x)
#pragma unroll
                        for (int v = 0; v < M; ++v) A[t][x][v] = u[x][v] + dtT * (O.xi[t] * R1[x][v]);
                it0 = 0;
            } else if (EX && S.guess == 4) {
                if constexpr (EX) {
                    // CERK guess (Sec. 2.2), stage by stage as in k_predictor
                    constexpr int CS = cerk_stages(N);
                    float w[n][M], Rk[n][M];
#pragma unroll
                    for (int t = 0; t < n; ++t)
#pragma unroll
                        for (int x = 0; x < n; ++x)
#pragma unroll
                            for (int v = 0; v < M; ++v) A[t][x][v] = u[x][v] + dtT * (O.ck_b[0][t] * R1[x][v]);
                    if constexpr (CS == 4) {
#pragma unroll
                        for (int x = 0; x < n; ++x)
#pragma unroll
                            for (int v = 0; v < M; ++v) w[x][v] = u[x][v] + 0.5f * dtT * R1[x][v];
#pragma unroll 1
                        for (int st = 1; st < 4; ++st) {
                            spatial_R(w, Rk);
#pragma unroll
                            for (int t = 0; t < n; ++t) {
                                const float bt = st == 3 ? O.ck_b[3][t] : O.ck_b[1][t];  // b2 = b3
#pragma unroll
                                for (int x = 0; x < n; ++x)
#pragma unroll
                                    for (int v = 0; v < M; ++v) A[t][x][v] += dtT * (bt * Rk[x][v]);
                            }
                            const float cs = st == 1 ? 0.5f : 1.0f;
#pragma unroll
                            for (int x = 0; x < n; ++x)
#pragma unroll
                                for (int v = 0; v < M; ++v) w[x][v] = u[x][v] + cs * dtT * Rk[x][v];
                        }
                    } else {
                        // the earlier stages' k of the row in registers (this
                        // kernel serves small rows: n^2 m <= 100)
                        float K[CS - 1][n][M];
#pragma unroll
                        for (int x = 0; x < n; ++x)
#pragma unroll
                            for (int v = 0; v < M; ++v) K[0][x][v] = R1[x][v];
#pragma unroll
                        for (int st = 1; st < CS; ++st) {
#pragma unroll
                            for (int x = 0; x < n; ++x)
#pragma unroll
                                for (int v = 0; v < M; ++v) {
                                    float acc = 0.f;
#pragma unroll
                                    for (int j = 0; j < st; ++j) acc += O.ck_a[st * (st - 1) / 2 + j] * K[j][x][v];
                                    w[x][v] = u[x][v] + dtT * acc;
                                }
                            spatial_R(w, Rk);
#pragma unroll
                            for (int t = 0; t < n; ++t) {
                                const float bt = O.ck_b[st][t];
#pragma unroll
                                for (int x = 0; x < n; ++x)
#pragma unroll
                                    for (int v = 0; v < M; ++v) A[t][x][v] += dtT * (bt * Rk[x][v]);
                            }
                            if (st < CS - 1) {
#pragma unroll
                                for (int x = 0; x < n; ++x)
#pragma unroll
                                    for (int v = 0; v < M; ++v) K[st][x][v] = Rk[x][v];
                            }
                        }
                    }
                }
                it0 = 0;
            } else {
#pragma unroll
                for (int t = 0; t < n; ++t)
#pragma unroll
                    for (int x = 0; x < n; ++x)
#pragma unroll
                        for (int v = 0; v < M; ++v) A[t][x][v] = u[x][v] + dtT * (O.c1[t] * R1[x][v]);
                it0 = 1;
            }
        }

        // ---- Picard iterations of eq. pde.st2 ------------------------------
        for (int it = it0; it < P_it; ++it) {
#pragma unroll
            for (int t = 0; t < n; ++t) {
                float Fx[n][M];
                float Sx[PDE::HAS_SRC ? n : 1][M];  // dx_0 S(q) of the row, before A[t] becomes R
#pragma unroll
                for (int x = 0; x < n; ++x) {
                    float F[2][M];
                    PDE::flux_delta(P.pde, ref, A[t][x], F);
#pragma unroll
                    for (int v = 0; v < M; ++v) Fx[x][v] = F[0][v];
                    if (act) IO::store(eb + ((t * n + y) * n + x) * M, F[1]);
                    if constexpr (PDE::HAS_SRC) {
#pragma unroll
                        for (int v = 0; v < M; ++v) Sx[x][v] = 0.f;
                        add_src(A[t][x], Sx[x]);
                    }
                }
                xt_contract_x<n, M>(Fx, A[t], Dm);
                if constexpr (PDE::HAS_SRC) {
#pragma unroll
                    for (int x = 0; x < n; ++x)
#pragma unroll
                        for (int v = 0; v < M; ++v) A[t][x][v] += Sx[x][v];
                }
            }
            __syncthreads();
            if (act) {
#pragma unroll
                for (int t = 0; t < n; ++t) xt_contract_y<n, M>(eb, t, y, Dm);
            }
            __syncthreads();
#pragma unroll
            for (int t = 0; t < n; ++t)
#pragma unroll
                for (int x = 0; x < n; ++x) {
                    float r[M];
                    IO::load(eb + ((t * n + y) * n + x) * M, r);
#pragma unroll
                    for (int v = 0; v < M; ++v) A[t][x][v] += ratio1 * r[v];
                }
            __syncthreads();  // eb is rewritten by the next iteration
            // q[t] = u + dt/dx_0 sum_t' iK1W[t][t'] R[t'], column by column
#pragma unroll
            for (int x = 0; x < n; ++x) {
                float Rc[n][M];
#pragma unroll
                for (int t = 0; t < n; ++t)
#pragma unroll
                    for (int v = 0; v < M; ++v) Rc[t][v] = A[t][x][v];
#pragma unroll
                for (int v = 0; v < M; ++v)
#pragma unroll
                    for (int t = 0; t < n; ++t) {
                        float acc = O.iK1W[t * n] * Rc[0][v];
#pragma unroll
                        for (int tp = 1; tp < n; ++tp) acc += O.iK1W[t * n + tp] * Rc[tp][v];
                        A[t][x][v] = u[x][v] + dtT * acc;
                    }
            }
        }

        if constexpr (EX) {
            if (S.guess == 3 && valid) {  // this step's predictor, for the next step's guess
                float *qp = reinterpret_cast<float *>(S.qprev) + ec * (n * NS * M);
#pragma unroll
                for (int t = 0; t < n; ++t)
#pragma unroll
                    for (int x = 0; x < n; ++x) IO::store(qp + (t * NS + y * n + x) * M, A[t][x]);
            }
        }

        // ---- time averages qbar, Fbar_x (registers), Fbar_y (shared) -------
        float *sQ = eb;             // qbar   [y][x][v]
        float *sFy = eb + NS * M;   // Fbar_y [y][x][v]
        float qb[n][M], fbx[n][M];
#pragma unroll
        for (int x = 0; x < n; ++x) {
            float fby[M];
#pragma unroll
            for (int v = 0; v < M; ++v) { qb[x][v] = 0.f; fbx[x][v] = 0.f; fby[v] = 0.f; }
#pragma unroll
            for (int t = 0; t < n; ++t) {
                float F[2][M];
                PDE::flux_delta(P.pde, ref, A[t][x], F);
                const float wt = O.w[t];
#pragma unroll
                for (int v = 0; v < M; ++v) {
                    qb[x][v] += wt * A[t][x][v];
                    fbx[x][v] += wt * F[0][v];
                    fby[v] += wt * F[1][v];
                }
            }
            if (act) {
                IO::store(sQ + (y * n + x) * M, qb[x]);
                IO::store(sFy + (y * n + x) * M, fby);
            }
        }
        __syncthreads();

        if (valid) {
            // ---- volume term V = (1/dx_0) Kw Fbar_x + (1/dx_1) Kw Fbar_y ------
            float *Vout = reinterpret_cast<float *>(S.V) + ec * (NS * M);
            const float *Ky = sKw + y * n;
#pragma unroll
            for (int x = 0; x < n; ++x) {
                float ax[M], ay[M], Vn[M];
#pragma unroll
                for (int v = 0; v < M; ++v) { ax[v] = 0.f; ay[v] = 0.f; }
#pragma unroll
                for (int j = 0; j < n; ++j) {
                    const float kx = O.Kv[0][x * n + j];
#pragma unroll
                    for (int v = 0; v < M; ++v) ax[v] += kx * fbx[j][v];
                }
#pragma unroll
                for (int j = 0; j < n; ++j) {
                    float f[M];
                    IO::load(sFy + (j * n + x) * M, f);
                    const float ky = Ky[j];
#pragma unroll
                    for (int v = 0; v < M; ++v) ay[v] += ky * f[v];
                }
#pragma unroll
                for (int v = 0; v < M; ++v) Vn[v] = idx0 * ax[v] + idx1 * ay[v];
                if constexpr (PDE::HAS_SRC) {  // S linear: its time average is S(qbar)
                    float qa[M], Sq[M];
#pragma unroll
                    for (int v = 0; v < M; ++v) qa[v] = qb[x][v] + ref.q[v];
                    PDE::source(P.pde, qa, Sq);
#pragma unroll
                    for (int v = 0; v < M; ++v) Vn[v] += Sq[v];
                }
                IO::store(Vout + (y * n + x) * M, Vn);
            }

            // ---- face traces: x faces at p = y (registers), y faces at p = x = y
            float *trE = reinterpret_cast<float *>(S.tr) + ec * (NREC * RS);
#pragma unroll
            for (int side = 0; side < 2; ++side) {
                const float *phi = side ? O.F1 : O.F0;
                float aq[M], af[M], full[M];
#pragma unroll
                for (int v = 0; v < M; ++v) { aq[v] = 0.f; af[v] = 0.f; }
#pragma unroll
                for (int j = 0; j < n; ++j)
#pragma unroll
                    for (int v = 0; v < M; ++v) {
                        aq[v] += phi[j] * qb[j][v];
                        af[v] += phi[j] * fbx[j][v];
                    }
                float *rec = trE + ((0 * 2 + side) * NF + y) * RS;
#pragma unroll
                for (int v = 0; v < M; ++v) {
                    rec[v] = aq[v];
                    rec[M + v] = af[v];
                    full[v] = aq[v] + ref.q[v];
                }
                rec[2 * M] = PDE::max_eig(P.pde, full, 0);
                rec[2 * M + 1] = 0.f;
            }
#pragma unroll
            for (int side = 0; side < 2; ++side) {
                const float *phi = side ? sF1 : sF0;
                float aq[M], af[M], full[M];
#pragma unroll
                for (int v = 0; v < M; ++v) { aq[v] = 0.f; af[v] = 0.f; }
#pragma unroll
                for (int j = 0; j < n; ++j) {
                    float qj[M], fj[M];
                    IO::load(sQ + (j * n + y) * M, qj);
                    IO::load(sFy + (j * n + y) * M, fj);
                    const float pj = phi[j];
#pragma unroll
                    for (int v = 0; v < M; ++v) {
                        aq[v] += pj * qj[v];
                        af[v] += pj * fj[v];
                    }
                }
                float *rec = trE + ((1 * 2 + side) * NF + y) * RS;
#pragma unroll
                for (int v = 0; v < M; ++v) {
                    rec[v] = aq[v];
                    rec[M + v] = af[v];
                    full[v] = aq[v] + ref.q[v];
                }
                rec[2 * M] = PDE::max_eig(P.pde, full, 1);
                rec[2 * M + 1] = 0.f;
            }
            if (y == 0) {  // the reference state, kept in FP64 for the corrector
#pragma unroll
                for (int v = 0; v < M; ++v) S.ref[ec * C::RF + v] = uref[v];
            }
        }
        // eb (and sDt) are rewritten by the next tile after its first barrier
    }
}
