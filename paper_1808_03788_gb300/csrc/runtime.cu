// Solver runtime behind the C ABI of include/aderdg.h: handle creation,
// device buffers, the per-step launch sequence (dt -> predictor ->
// corrector), CUDA-graph replay for multi-step advances, and the small
// generic kernels (CFL step, conserved totals, trace unpacking).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/aderdg.h"
#include "basis.h"
#include "common.cuh"
#include "control.cuh"
#include "tune.h"


using namespace aderdg;

namespace {

thread_local std::string g_err = "no error";

int fail(int code, const std::string &msg)
{
    g_err = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char *what)
{
    return fail(ADERDG_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                        \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

const KernelSet *find_kernels(int pde, int dim, int N, int prec)
{
    return lookup_kernels(pde, dim, N, prec);
}


// ---------------------------------------------------------------------------
// generic kernels
// ---------------------------------------------------------------------------

// CFL step of Sec. 3 for the handle's solve (control.cuh).
__global__ void k_dt(Control *c)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    dt_update(c);
}

// dt the CFL condition gives for the current maxima (no clip, no update).
__global__ void k_cfl_query(const Control *c, double *out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double S = 0.0;
    for (int d = 0; d < c->dim; ++d) S += __longlong_as_double((long long)c->lam_acc[d]) * c->inv_dx[d];
    out[0] = c->alpha / S;
}

// Conserved totals, stage 1: block b sums the elements b, b + G, b + 2G, ...
// per thread in a fixed order, then a fixed-shape tree per block.
constexpr int MASS_THREADS = 256;
constexpr int MASS_BLOCKS = 304;

__global__ void __launch_bounds__(MASS_THREADS)
k_mass_partial(const double *u, long long E, int NS, int M, int n, int dim, Basis b, double vol,
               double *partial)
{
    __shared__ double red[MASS_THREADS * 9];
    double acc[9];
    for (int v = 0; v < 9; ++v) acc[v] = 0.0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < E; e += stride) {
        for (int s = 0; s < NS; ++s) {
            double ws = vol;
            int r = s;
            for (int d = 0; d < dim; ++d) { ws *= b.w[r % n]; r /= n; }
            for (int v = 0; v < M; ++v) acc[v] += ws * u[(e * NS + s) * M + v];
        }
    }
    for (int v = 0; v < M; ++v) red[threadIdx.x * 9 + v] = acc[v];
    __syncthreads();
    for (int h = MASS_THREADS / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h)
            for (int v = 0; v < M; ++v) red[threadIdx.x * 9 + v] += red[(threadIdx.x + h) * 9 + v];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int v = 0; v < M; ++v) partial[blockIdx.x * 9 + v] = red[v];
}

__global__ void k_mass_final(const double *partial, int nb, int M, double *out)
{
    const int v = threadIdx.x;
    if (v >= M) return;
    double s = 0.0;
    for (int i = 0; i < nb; ++i) s += partial[i * 9 + v];
    out[v] = s;
}

// Predictor trace records [e][d][side][p][RS] (T) -> oracle layout
// qface/fface [e][d][side][p][v] (double).
template <typename T>
__global__ void k_unpack_traces(const T *tr, long long nrec_total, int M, int RS, int has_flux, double *qf,
                                double *ff)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= nrec_total * M) return;
    const long long r = i / M;
    const int v = (int)(i - r * M);
    if (qf) qf[i] = double(tr[r * RS + v]);
    if (ff) ff[i] = has_flux ? double(tr[r * RS + M + v]) : 0.0;  // no flux in purely non-conservative records
}

template <typename T>
__global__ void k_widen(const T *src, long long count, double *dst)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < count) dst[i] = double(src[i]);
}

}  // namespace

namespace aderdg {
// lets other translation units of the library report through aderdg_last_error
void set_last_error(const char *msg) { g_err = msg; }
}  // namespace aderdg

// ---------------------------------------------------------------------------
// the handle
// ---------------------------------------------------------------------------

struct aderdg_s {
    int dim = 0, N = 0, n = 0, M = 0, pde = 0, precision = 0, picard = 0, guess = 0;
    long long E = 0;
    int NS = 0, NF = 0, NREC = 0;
    double dx[3] = {1, 1, 1};
    double lo[3] = {0, 0, 0}, hi[3] = {1, 1, 1};
    double alpha = 0;
    const KernelSet *ks = nullptr;  // = &kso
    KernelSet kso{};                // kernels with the tile shapes in use
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    aderdg_alloc_t alloc{};
    bool has_alloc = false;
    double *u = nullptr;
    void *V = nullptr;
    void *tr = nullptr;
    Control *ctl = nullptr;
    double *scratch = nullptr;  // mass partials + small outputs
    double *ref = nullptr;      // FP32 path: per-element reference records
    void *qprev = nullptr;      // extrapolation guess: last predictor [E][n][NS][M]
    bool limiter = false;       // subcell limiter after every step
    LimKernels lk{};            // its kernels
    double *u_prev = nullptr;   // limiter: u^n saved before the corrector
    double *lim_mm = nullptr;   // limiter: extreme subcell averages of u^n [E][M][2]
    double *lim_mmc = nullptr;  // limiter: those of the candidate, kept for the next step
    int *lim_flags = nullptr;   // limiter: troubled elements of the last step [E]
    int *lim_list = nullptr;    // limiter: their indices, in detection order [E]
    bool lim_keep = false;      // limiter: subcell data of limited elements kept between steps
    int NSUB = 0;               // subcells per element, (2N+1)^d
    double *lim_sub = nullptr;  // kept: subcell data of u^n [E][NSUB][M]
    double *lim_subn = nullptr; // kept: new averages of the step's troubled elements [E][NSUB][M]
    int *lim_kept = nullptr;    // kept: lim_sub[e] holds e's subcell data of u^n [E]
    double *lim_fb = nullptr;   // limiter: troubled elements' face fluxes for the coupling
    int *lim_slot = nullptr;    // limiter: their slots [E]
    long long lim_fb_slots = 0;
    double *host_pinned = nullptr;
    KParams kp{};
    Basis basis{};
    SolveDesc desc{};             // host copy of the single solve's descriptor
    SolveDesc *d_desc = nullptr;  // device copy
    double inv_dx[3] = {1, 1, 1};
    size_t device_bytes = 0;
    cudaGraphExec_t graph = nullptr;
    int graph_steps = 0;
    int device = 0;
    bool profiling = false;
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    // limiter: the copy of u^n and its subcell extremes run on a second
    // stream while the predictor runs (forked and joined by events, so a
    // stream capture takes both branches)
    cudaStream_t side = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
};

namespace {

void *dev_alloc(aderdg_t *h, size_t bytes)
{
    void *p = nullptr;
    bytes = (bytes + 255) / 256 * 256;
    if (h->has_alloc) p = h->alloc.alloc(bytes, h->alloc.ctx);
    else if (cudaMalloc(&p, bytes) != cudaSuccess) p = nullptr;
    if (p) h->device_bytes += bytes;
    return p;
}

void dev_free(aderdg_t *h, void *p)
{
    if (!p) return;
    if (h->has_alloc) h->alloc.free(p, h->alloc.ctx);
    else cudaFree(p);
}

int launch_predictor(aderdg_t *h, int use_ctl, double dt)
{
    KParams kp = h->kp;
    kp.use_ctl_dt = use_ctl;
    kp.dt_arg = dt;
    kp.ntiles = (h->E + h->ks->pred_epb - 1) / h->ks->pred_epb;
    h->ks->predictor<<<(unsigned)kp.ntiles, h->ks->pred_threads, h->ks->pred_smem, h->stream>>>(kp);
    CK(cudaGetLastError());
    return ADERDG_OK;
}

int launch_corrector(aderdg_t *h, int use_ctl, double dt)
{
    KParams kp = h->kp;
    kp.use_ctl_dt = use_ctl;
    kp.dt_arg = dt;
    kp.ntiles = (h->E + h->ks->corr_epb - 1) / h->ks->corr_epb;
    h->ks->corrector<<<(unsigned)kp.ntiles, h->ks->corr_threads, h->ks->corr_smem, h->stream>>>(kp);
    CK(cudaGetLastError());
    return ADERDG_OK;
}


// The subcell limiter on the candidate the corrector left in u (Sec. 2.3):
// detection, subcell finite-volume update of the troubled elements,
// coupling of their unlimited neighbours, and the wave-speed maxima of the
// limited state for the next CFL step.
// The extremes of u^n's subcell averages (the maximum principle's bounds);
// they read u_prev only, so the step runs them beside the predictor.
int launch_lim_minmax(aderdg_t *h, cudaStream_t st)
{
    KParams kp = h->kp;
    kp.use_ctl_dt = 1;
    h->lk.minmax<<<h->lk.minmax_grid(h->E), 128, h->lk.smem_w, st>>>(kp);
    CK(cudaGetLastError());
    return ADERDG_OK;
}

int launch_limiter(aderdg_t *h)
{
    const KernelSet *ks = h->ks;
    KParams kp = h->kp;
    kp.use_ctl_dt = 1;
    const LimKernels &lk = h->lk;
    const unsigned grid = (unsigned)std::min<long long>(h->E, 152LL * 16);
    lk.detect<<<grid, 128, lk.smem_w, h->stream>>>(kp);
    lk.fv<<<grid, 128, lk.smem, h->stream>>>(kp);
    lk.couple<<<grid, 128, lk.smem, h->stream>>>(kp);
    kp.lim_pass = 1;  // the wave speeds of the limited state, if it changed
    ks->cfl<<<(unsigned)std::min<long long>(4 * 152, (h->E * h->NS + 255) / 256), 256, 0, h->stream>>>(kp);
    CK(cudaGetLastError());
    return ADERDG_OK;
}

int enqueue_step(aderdg_t *h)
{
    k_dt<<<1, 32, 0, h->stream>>>(h->ctl);
    CK(cudaGetLastError());
    if (h->limiter) {
        // u^n saved and its subcell extremes formed on the side stream, in
        // the predictor's shadow (both read u^n, which the predictor does not
        // write); the corrector, which overwrites u, waits for them
        CK(cudaEventRecord(h->fork, h->stream));
        CK(cudaStreamWaitEvent(h->side, h->fork, 0));
        CK(cudaMemcpyAsync(h->u_prev, h->u, (size_t)h->E * h->NS * h->M * sizeof(double), cudaMemcpyDeviceToDevice,
                           h->side));
        int rc = launch_lim_minmax(h, h->side);
        if (rc) return rc;
        CK(cudaEventRecord(h->join, h->side));
    }
    if (h->profiling) CK(cudaEventRecord(h->ev[0], h->stream));
    int rc = launch_predictor(h, 1, 0.0);
    if (rc) return rc;
    if (h->limiter) CK(cudaStreamWaitEvent(h->stream, h->join, 0));
    if (h->profiling) CK(cudaEventRecord(h->ev[1], h->stream));
    rc = launch_corrector(h, 1, 0.0);
    if (rc) return rc;
    if (h->profiling) CK(cudaEventRecord(h->ev[2], h->stream));
    if (h->limiter) return launch_limiter(h);
    return ADERDG_OK;
}

int read_ctl(aderdg_t *h, Control *out)
{
    CK(cudaMemcpyAsync(h->host_pinned, h->ctl, sizeof(Control), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    std::memcpy(out, h->host_pinned, sizeof(Control));
    return ADERDG_OK;
}

int check_flags(const Control &c)
{
    if (c.flags & FLAG_NONFINITE) return fail(ADERDG_E_NONFINITE, "non-finite value in the state");
    if (c.flags & FLAG_TIMEOUT) return fail(ADERDG_E_TIMEOUT, "bounded device wait expired");
    return ADERDG_OK;
}

int set_t_end(aderdg_t *h, double t_end)
{
    std::memcpy(h->host_pinned + 64, &t_end, sizeof(double));
    CK(cudaMemcpyAsync(&h->ctl->t_end, h->host_pinned + 64, sizeof(double), cudaMemcpyHostToDevice,
                       h->stream));
    // the pinned staging slot is reused: wait until the copy has read it
    CK(cudaStreamSynchronize(h->stream));
    return ADERDG_OK;
}

// Algorithmic counts of the kernels as formulated (FMA = 2 flops; a
// reciprocal or square root = 1): the initial guess (trivial: the first
// Picard iteration on the time-constant guess, then P-1 full iterations;
// second / third order: one / two time-constant L evaluations, then P full
// iterations; extrapolation: an n x n contraction per node and variable,
// then P full iterations, with the previous predictor read and this one
// written), time averages, volume term, traces; corrector Rusanov +
// lift + update + wave speeds.
void fill_cost(const aderdg_t *h, aderdg_info_t *info)
{
    const double n = h->n, M = h->M, NS = h->NS, NST = h->NS * h->n, NF = h->NF, NREC = h->NREC, D = h->dim;
    const double P = h->picard, FF = h->ks->flux_flops, EF = h->ks->eig_flops;
    const double MX = h->ks->mx;  // variables whose derivatives are taken (all m, or fewer for B-only systems)
    const double it1 = NS * FF + D * NF * MX * 2 * n * n + NS * MX * (D - 1) + n * NS * M * 3;
    const double itk = NST * FF + D * NS * MX * 2 * n * n + NST * MX * (D - 1) + NS * M * n * (2 * n + 2);
    // a purely non-conservative system averages q only and takes its volume
    // term as one more L evaluation on qbar (it1 without the time expansion)
    const double fin = h->ks->ncp ? NST * M * 2 + (it1 - n * NS * M * 3) + NS * M + NREC * M * 2 * n + NREC * EF
                                  : NST * FF + (1 + D) * NST * M * 2 + NS * M * D * 2 * n + NREC * M * 4 * n +
                                        NREC * EF;
    double pred;
    if (h->guess == 3) pred = NST * M * 2 * n + P * itk + fin;  // steady state (a previous predictor)
    else if (h->guess == 4) {  // S stages; the classical method forms each stage state with one product
        const double S = cerk_stages(h->N);
        pred = S * it1 + (S == 4 ? 6.0 : S * (S - 1)) * NS * M + P * itk + fin;
    }
    else if (h->guess == 2) pred = 2 * it1 + 2 * NS * M + P * itk + fin;  // it1 counts 3 flops per q value, the
                                                                     // Taylor form 6 over two evaluations
    else if (h->guess == 1) pred = it1 + P * itk + fin;
    else pred = it1 + (P - 1) * itk + fin;
    double corr = NREC * M * 6 + NREC + NS * M * (5 * D + 3) + NS * D * (EF + 1);
    if (h->ks->ncp) corr += NREC * 3 * (FF / D + 2 * M);  // three-point path integral per record
    info->flops_predictor = pred * h->E;
    info->flops_corrector = corr * h->E;
    const double b = h->ks->elem_bytes;
    info->bytes_predictor = h->E * (8.0 * NS * M + b * NS * M + b * NREC * h->ks->rs);
    if (h->guess == 3) info->bytes_predictor += h->E * 2.0 * b * NST * M;  // previous predictor in, this one out
    info->bytes_corrector = h->E * (16.0 * NS * M + b * NS * M + 2.0 * b * NREC * h->ks->rs);
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

extern "C" {

const char *aderdg_last_error(void) { return g_err.c_str(); }

int aderdg_version(void) { return 100; }

int aderdg_gl_nodes(int N, double *x, double *w)
{
    if (N < 1 || N > 9 || !x || !w) return fail(ADERDG_E_INVAL, "aderdg_gl_nodes: need 1 <= N <= 9");
    if (gauss_legendre01(N + 1, x, w)) return fail(ADERDG_E_INVAL, "gauss_legendre01 failed");
    return ADERDG_OK;
}

double aderdg_default_alpha(int N) { return default_alpha(N); }

int aderdg_create(const aderdg_mesh_t *mesh, int N, int nVar, const aderdg_pde_t *pde,
                  const aderdg_config_t *cfg, aderdg_t **out)
{
    if (!out) return fail(ADERDG_E_INVAL, "out is NULL");
    *out = nullptr;
    if (!mesh || !pde) return fail(ADERDG_E_INVAL, "mesh/pde is NULL");
    long long E = 0;
    const char *why = nullptr;
    if (check_mesh(*mesh, pde->kind, &E, &why)) return fail(ADERDG_E_INVAL, why);
    const int m = pde_nvar(pde->kind, mesh->dim);
    if (nVar != m) return fail(ADERDG_E_INVAL, "nVar does not match the PDE");
    if (N < 1 || N > 9) return fail(ADERDG_E_INVAL, "N must be in 1..9");
    const int prec = cfg ? cfg->precision : ADERDG_FP64;
    if (prec != ADERDG_FP64 && prec != ADERDG_MIXED_FP32) return fail(ADERDG_E_INVAL, "bad precision");
    const KernelSet *ks = find_kernels(pde->kind, mesh->dim, N, prec);
    if (!ks) return fail(ADERDG_E_UNSUPPORTED, "no kernels compiled for this (pde, dim, N)");
    if (check_pde_params(*pde, &why)) return fail(ADERDG_E_INVAL, why);

    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return fail(ADERDG_E_CUDA, "no CUDA device available (the library has no CPU path)");
    }

    aderdg_t *h = new aderdg_s();
    cudaGetDevice(&h->device);
    h->dim = mesh->dim;
    h->N = N;
    h->n = N + 1;
    h->M = m;
    h->pde = pde->kind;
    h->precision = prec;
    h->guess = cfg ? cfg->initial_guess : ADERDG_GUESS_TRIVIAL;
    if (h->guess < ADERDG_GUESS_TRIVIAL || h->guess > ADERDG_GUESS_CERK) {
        delete h;
        return fail(ADERDG_E_INVAL, "bad initial guess");
    }
    if (cfg && (cfg->limiter < 0 || cfg->limiter > 2)) {
        delete h;
        return fail(ADERDG_E_INVAL, "limiter must be 0, 1 or 2");
    }
    h->limiter = cfg && cfg->limiter;
    h->lim_keep = cfg && cfg->limiter == 2;
    if (h->limiter) {
        const int rc = limiter_kernels(pde->kind, mesh->dim, N, prec, h->guess, h->lim_keep, &h->lk, &why);
        if (rc) {
            delete h;
            return fail(rc, why);
        }
    }
    h->picard = (cfg && cfg->picard_iters > 0) ? cfg->picard_iters : default_picard(N, h->guess);
    h->alpha = (cfg && cfg->cfl_alpha > 0) ? cfg->cfl_alpha : default_alpha(N);
    h->E = E;
    h->NS = ipow(h->n, h->dim);
    h->NF = ipow(h->n, h->dim - 1);
    h->NREC = h->dim * 2 * h->NF;
    {
        PdeParams pp;
        for (int i = 0; i < 8; ++i) pp.p[i] = pde->p[i];
        fill_pde_consts(pde->kind, pp);
        const int rc = resolve_shapes(ks, pde->kind, mesh->dim, N, prec, pp, cfg ? cfg->pred_shape : 0,
                                      cfg ? cfg->corr_shape : 0, cfg ? cfg->tune_cache : nullptr,
                                      h->guess == ADERDG_GUESS_EXTRAP || h->guess == ADERDG_GUESS_CERK, &h->kso);
        if (rc) { delete h; return rc; }
    }
    h->ks = ks = &h->kso;
    for (int d = 0; d < 3; ++d) {
        h->lo[d] = d < h->dim ? mesh->lo[d] : 0.0;
        h->hi[d] = d < h->dim ? mesh->hi[d] : 1.0;
        h->dx[d] = d < h->dim ? (mesh->hi[d] - mesh->lo[d]) / mesh->cells[d] : 1.0;
    }
    if (cfg && cfg->alloc) {
        if (!cfg->alloc->alloc || !cfg->alloc->free) { delete h; return fail(ADERDG_E_INVAL, "allocator incomplete"); }
        h->alloc = *cfg->alloc;
        h->has_alloc = true;
    }
    if (cfg && cfg->cuda_stream) h->stream = (cudaStream_t)cfg->cuda_stream;
    else {
        if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete h;
            return fail(ADERDG_E_CUDA, "cudaStreamCreate failed");
        }
        h->own_stream = true;
    }
    if (build_basis(N, h->basis)) { aderdg_destroy(h); return fail(ADERDG_E_INVAL, "basis construction failed"); }

    const size_t nstate = (size_t)E * h->NS * m;
    h->u = (double *)dev_alloc(h, nstate * sizeof(double));
    h->V = dev_alloc(h, nstate * ks->elem_bytes);
    h->tr = dev_alloc(h, (size_t)E * h->NREC * ks->rs * ks->elem_bytes);
    h->ctl = (Control *)dev_alloc(h, sizeof(Control));
    h->scratch = (double *)dev_alloc(h, sizeof(double) * (MASS_BLOCKS * 9 + 64));
    h->d_desc = (SolveDesc *)dev_alloc(h, sizeof(SolveDesc));
    if (ks->rf > 0) h->ref = (double *)dev_alloc(h, sizeof(double) * (size_t)E * ks->rf);
    if (h->guess == ADERDG_GUESS_EXTRAP) h->qprev = dev_alloc(h, nstate * h->n * ks->elem_bytes);
    if (h->limiter) {
        h->u_prev = (double *)dev_alloc(h, nstate * sizeof(double));
        h->lim_mm = (double *)dev_alloc(h, sizeof(double) * (size_t)E * m * 2);
        h->lim_mmc = (double *)dev_alloc(h, sizeof(double) * (size_t)E * m * 2);
        h->lim_flags = (int *)dev_alloc(h, sizeof(int) * (size_t)E);
        h->lim_list = (int *)dev_alloc(h, sizeof(int) * (size_t)E);
    }
    h->NSUB = ipow(2 * N + 1, h->dim);
    if (h->limiter) {
        h->lim_fb_slots = limiter_flux_slots(E, h->dim, N, m, ks->ncp != 0);
        if (h->lim_fb_slots > 0) {
            h->lim_fb = (double *)dev_alloc(
                h, sizeof(double) * (size_t)h->lim_fb_slots * limiter_flux_doubles(h->dim, N, m, ks->ncp != 0));
            h->lim_slot = (int *)dev_alloc(h, sizeof(int) * (size_t)E);
        }
    }
    if (h->lim_keep) {
        h->lim_sub = (double *)dev_alloc(h, sizeof(double) * (size_t)E * h->NSUB * m);
        h->lim_subn = (double *)dev_alloc(h, sizeof(double) * (size_t)E * h->NSUB * m);
        h->lim_kept = (int *)dev_alloc(h, sizeof(int) * (size_t)E);
    }
    if (!h->u || !h->V || !h->tr || !h->ctl || !h->scratch || !h->d_desc || (ks->rf > 0 && !h->ref) ||
        (h->guess == ADERDG_GUESS_EXTRAP && !h->qprev) ||
        (h->limiter && (!h->u_prev || !h->lim_mm || !h->lim_mmc || !h->lim_flags || !h->lim_list)) ||
        (h->lim_keep && (!h->lim_sub || !h->lim_subn || !h->lim_kept)) ||
        (h->lim_fb_slots > 0 && (!h->lim_fb || !h->lim_slot))) {
        aderdg_destroy(h);
        return fail(ADERDG_E_NOMEM, "device allocation failed");
    }
    if (cudaMallocHost(&h->host_pinned, 4096) != cudaSuccess) {
        h->host_pinned = nullptr;
        aderdg_destroy(h);
        return fail(ADERDG_E_NOMEM, "pinned host allocation failed");
    }
    if (h->limiter && (cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking) != cudaSuccess ||
                       cudaEventCreateWithFlags(&h->fork, cudaEventDisableTiming) != cudaSuccess ||
                       cudaEventCreateWithFlags(&h->join, cudaEventDisableTiming) != cudaSuccess)) {
        aderdg_destroy(h);
        return fail(ADERDG_E_CUDA, "limiter stream or events");
    }

    SolveDesc &sd = h->desc;
    std::memset(&sd, 0, sizeof(sd));
    sd.E = E;
    for (int d = 0; d < 3; ++d) {
        sd.cells[d] = d < h->dim ? (int)mesh->cells[d] : 1;
        h->inv_dx[d] = 1.0 / h->dx[d];
        sd.inv_dx[d] = h->inv_dx[d];
    }
    fill_desc_spacing(sd);
    fill_desc_lift(sd, N);
    sd.picard = h->picard;
    sd.guess = h->guess;
    sd.picard_first = default_picard(N, ADERDG_GUESS_ORDER3);
    sd.qprev = h->qprev;
    sd.u = h->u;
    sd.u_out = h->u;
    sd.V = h->V;
    sd.tr = h->tr;
    sd.ref = h->ref;
    sd.ctl = h->ctl;
    sd.u_prev = h->u_prev;
    sd.lim_mm = h->lim_mm;
    sd.lim_mmc = h->lim_mmc;
    sd.lim_flags = h->lim_flags;
    sd.lim_list = h->lim_list;
    sd.lim_sub = h->lim_sub;
    sd.lim_subn = h->lim_subn;
    sd.lim_kept = h->lim_kept;
    sd.lim_fb = h->lim_fb;
    sd.lim_slot = h->lim_slot;
    sd.lim_fb_slots = h->lim_fb_slots;
    KParams &kp = h->kp;
    std::memset(&kp, 0, sizeof(kp));
    kp.solves = h->d_desc;
    kp.nsolves = 1;
    for (int i = 0; i < 8; ++i) kp.pde.p[i] = pde->p[i];
    fill_pde_consts(pde->kind, kp.pde);
    kp.b = h->basis;
    fill_ops(kp);

    Control c;
    std::memset(&c, 0, sizeof(c));
    c.alpha = h->alpha;
    c.dim = h->dim;
    for (int d = 0; d < 3; ++d) c.inv_dx[d] = h->inv_dx[d];
    c.t_end = 0.0;
    if (cudaMemcpyAsync(h->d_desc, &sd, sizeof(sd), cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
        cudaMemsetAsync(h->u, 0, nstate * sizeof(double), h->stream) != cudaSuccess ||
        (h->limiter && cudaMemsetAsync(h->lim_flags, 0, sizeof(int) * (size_t)E, h->stream) != cudaSuccess) ||
        cudaMemcpyAsync(h->ctl, &c, sizeof(c), cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess) {
        aderdg_destroy(h);
        return fail(ADERDG_E_CUDA, "initialisation failed");
    }
    *out = h;
    return ADERDG_OK;
}

int aderdg_destroy(aderdg_t *h)
{
    if (!h) return ADERDG_OK;
    if (h->stream) cudaStreamSynchronize(h->stream);
    if (h->graph) cudaGraphExecDestroy(h->graph);
    dev_free(h, h->u);
    dev_free(h, h->u_prev);
    dev_free(h, h->lim_mm);
    dev_free(h, h->lim_mmc);
    dev_free(h, h->lim_flags);
    dev_free(h, h->lim_list);
    dev_free(h, h->lim_sub);
    dev_free(h, h->lim_subn);
    dev_free(h, h->lim_kept);
    dev_free(h, h->lim_fb);
    dev_free(h, h->lim_slot);
    dev_free(h, h->V);
    dev_free(h, h->tr);
    dev_free(h, h->ctl);
    dev_free(h, h->scratch);
    dev_free(h, h->d_desc);
    dev_free(h, h->ref);
    dev_free(h, h->qprev);
    if (h->host_pinned) cudaFreeHost(h->host_pinned);
    for (auto &e : h->ev)
        if (e) cudaEventDestroy(e);
    if (h->fork) cudaEventDestroy(h->fork);
    if (h->join) cudaEventDestroy(h->join);
    if (h->side) cudaStreamDestroy(h->side);
    if (h->own_stream) cudaStreamDestroy(h->stream);
    delete h;
    return ADERDG_OK;
}

int aderdg_get_info(const aderdg_t *h, aderdg_info_t *info)
{
    if (!h || !info) return fail(ADERDG_E_INVAL, "NULL argument");
    std::memset(info, 0, sizeof(*info));
    info->dim = h->dim;
    info->N = h->N;
    info->nvar = h->M;
    info->precision = h->precision;
    info->picard_iters = h->picard;
    info->initial_guess = h->guess;
    info->elements = h->E;
    info->dofs = h->E * h->NS;
    info->cfl_alpha = h->alpha;
    info->device_bytes = h->device_bytes;
    info->pred_shape = h->ks->pred_shape;
    info->pred_threads = h->ks->pred_threads;
    info->pred_epb = h->ks->pred_epb;
    info->corr_shape = h->ks->corr_shape;
    info->corr_threads = h->ks->corr_threads;
    info->corr_epb = h->ks->corr_epb;
    fill_cost(h, info);
    return ADERDG_OK;
}

int aderdg_set_state(aderdg_t *h, const double *u, int where, double t)
{
    if (!h || !u) return fail(ADERDG_E_INVAL, "NULL argument");
    if (!std::isfinite(t)) return fail(ADERDG_E_INVAL, "t must be finite");
    const size_t bytes = (size_t)h->E * h->NS * h->M * sizeof(double);
    CK(cudaMemcpyAsync(h->u, u, bytes, where == ADERDG_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                       h->stream));
    Control c;
    std::memset(&c, 0, sizeof(c));
    c.t = t;
    c.t_end = t;
    c.alpha = h->alpha;
    c.dim = h->dim;
    for (int d = 0; d < 3; ++d) c.inv_dx[d] = h->inv_dx[d];
    std::memcpy(h->host_pinned, &c, sizeof(c));
    CK(cudaMemcpyAsync(h->ctl, h->host_pinned, sizeof(c), cudaMemcpyHostToDevice, h->stream));
    h->ks->cfl<<<(unsigned)std::min<long long>(4 * 152, (h->E * h->NS + 255) / 256), 256, 0, h->stream>>>(h->kp);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(h->stream));  // the pinned staging buffer is reused
    return ADERDG_OK;
}

int aderdg_get_state(aderdg_t *h, double *u, int where, double *t, int64_t *step)
{
    if (!h || !u) return fail(ADERDG_E_INVAL, "NULL argument");
    const size_t bytes = (size_t)h->E * h->NS * h->M * sizeof(double);
    CK(cudaMemcpyAsync(u, h->u, bytes, where == ADERDG_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                       h->stream));
    Control c;
    int rc = read_ctl(h, &c);
    if (rc) return rc;
    if (t) *t = c.t;
    if (step) *step = c.step;
    return check_flags(c);
}

int aderdg_predictor(aderdg_t *h, double dt)
{
    if (!h) return fail(ADERDG_E_INVAL, "NULL handle");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(ADERDG_E_INVAL, "dt must be positive and finite");
    return launch_predictor(h, 0, dt);
}

int aderdg_corrector(aderdg_t *h, double dt)
{
    if (!h) return fail(ADERDG_E_INVAL, "NULL handle");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(ADERDG_E_INVAL, "dt must be positive and finite");
    CK(cudaMemsetAsync(h->ctl->lam_acc, 0, sizeof(h->ctl->lam_acc), h->stream));
    // the state changes without the limiter: its kept extremes and subcell
    // data are stale
    CK(cudaMemsetAsync(&h->ctl->lim_fresh, 0, sizeof(h->ctl->lim_fresh), h->stream));
    CK(cudaMemsetAsync(&h->ctl->lim_kept_ok, 0, sizeof(h->ctl->lim_kept_ok), h->stream));
    return launch_corrector(h, 0, dt);
}

int aderdg_set_subcell_state(aderdg_t *h, const double *avg, int where, double t)
{
    if (!h || !avg) return fail(ADERDG_E_INVAL, "NULL argument");
    if (!h->lim_keep) return fail(ADERDG_E_INVAL, "the handle does not keep subcell data (limiter 2)");
    if (!std::isfinite(t)) return fail(ADERDG_E_INVAL, "t must be finite");
    const size_t bytes = (size_t)h->E * h->NSUB * h->M * sizeof(double);
    CK(cudaMemcpyAsync(h->lim_subn, avg, bytes,
                       where == ADERDG_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream));
    Control c;
    std::memset(&c, 0, sizeof(c));
    c.t = t;
    c.t_end = t;
    c.alpha = h->alpha;
    c.dim = h->dim;
    for (int d = 0; d < 3; ++d) c.inv_dx[d] = h->inv_dx[d];
    std::memcpy(h->host_pinned, &c, sizeof(c));
    CK(cudaMemcpyAsync(h->ctl, h->host_pinned, sizeof(c), cudaMemcpyHostToDevice, h->stream));
    // the reconstruction of every element, all marked limited, then the
    // wave speeds of the subcell averages
    h->lk.init<<<(unsigned)std::min<long long>(h->E, 152LL * 16), 128, h->lk.smem, h->stream>>>(h->kp);
    CK(cudaGetLastError());
    h->ks->cfl<<<(unsigned)std::min<long long>(4 * 152, (h->E * h->NS + 255) / 256), 256, 0, h->stream>>>(h->kp);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(h->stream));  // the pinned staging buffer is reused
    return ADERDG_OK;
}

int aderdg_get_subcell_state(aderdg_t *h, double *avg, int where)
{
    if (!h || !avg) return fail(ADERDG_E_INVAL, "NULL argument");
    if (!h->lim_keep) return fail(ADERDG_E_INVAL, "the handle does not keep subcell data (limiter 2)");
    const size_t bytes = (size_t)h->E * h->NSUB * h->M * sizeof(double);
    CK(cudaMemcpyAsync(avg, h->lim_subn, bytes,
                       where == ADERDG_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return ADERDG_OK;
}

int aderdg_troubled(aderdg_t *h, int *flags, int64_t *count)
{
    if (!h) return fail(ADERDG_E_INVAL, "NULL handle");
    if (!h->limiter) return fail(ADERDG_E_INVAL, "the handle has no limiter");
    std::vector<int> f((size_t)h->E);
    CK(cudaMemcpyAsync(f.data(), h->lim_flags, sizeof(int) * (size_t)h->E, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    int64_t c = 0;
    for (long long e = 0; e < h->E; ++e) c += f[(size_t)e] != 0;
    if (flags) std::memcpy(flags, f.data(), sizeof(int) * (size_t)h->E);
    if (count) *count = c;
    return ADERDG_OK;
}

int aderdg_get_predictor_outputs(aderdg_t *h, double *volume, double *qface, double *fface, int where)
{
    if (!h) return fail(ADERDG_E_INVAL, "NULL handle");
    const long long nstate = h->E * h->NS * h->M;
    const long long nrec = h->E * h->NREC;
    const long long ntr = nrec * h->M;
    const int eb = h->ks->elem_bytes;
    double *tmp = nullptr;
    if (where != ADERDG_DEVICE) {
        const size_t need = sizeof(double) * (size_t)std::max(nstate, 2 * ntr);
        tmp = (double *)dev_alloc(h, need);
        if (!tmp) return fail(ADERDG_E_NOMEM, "temporary allocation failed");
    }
    int rc = ADERDG_OK;
    auto run = [&]() -> int {
        if (volume) {
            double *dst = where == ADERDG_DEVICE ? volume : tmp;
            const unsigned blocks = (unsigned)((nstate + 255) / 256);
            if (eb == 8) k_widen<double><<<blocks, 256, 0, h->stream>>>((const double *)h->V, nstate, dst);
            else k_widen<float><<<blocks, 256, 0, h->stream>>>((const float *)h->V, nstate, dst);
            CK(cudaGetLastError());
            if (where != ADERDG_DEVICE)
                CK(cudaMemcpyAsync(volume, tmp, nstate * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
            CK(cudaStreamSynchronize(h->stream));
        }
        if (qface || fface) {
            double *dq = where == ADERDG_DEVICE ? qface : (qface ? tmp : nullptr);
            double *df = where == ADERDG_DEVICE ? fface : (fface ? tmp + ntr : nullptr);
            const unsigned blocks = (unsigned)((ntr + 255) / 256);
            if (eb == 8)
                k_unpack_traces<double><<<blocks, 256, 0, h->stream>>>((const double *)h->tr, nrec, h->M, h->ks->rs,
                                                                       !h->ks->ncp, dq, df);
            else
                k_unpack_traces<float><<<blocks, 256, 0, h->stream>>>((const float *)h->tr, nrec, h->M, h->ks->rs,
                                                                      !h->ks->ncp, dq, df);
            CK(cudaGetLastError());
            if (where != ADERDG_DEVICE) {
                if (qface) CK(cudaMemcpyAsync(qface, dq, ntr * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
                if (fface) CK(cudaMemcpyAsync(fface, df, ntr * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
            }
            CK(cudaStreamSynchronize(h->stream));
        }
        return ADERDG_OK;
    };
    rc = run();
    if (tmp) {
        cudaStreamSynchronize(h->stream);
        dev_free(h, tmp);
        h->device_bytes -= (sizeof(double) * (size_t)std::max(nstate, 2 * ntr) + 255) / 256 * 256;
    }
    return rc;
}

int aderdg_step(aderdg_t *h, double t_end, double *dt_taken)
{
    if (!h) return fail(ADERDG_E_INVAL, "NULL handle");
    if (!std::isfinite(t_end)) return fail(ADERDG_E_INVAL, "t_end must be finite");
    int rc = set_t_end(h, t_end);
    if (rc) return rc;
    rc = enqueue_step(h);
    if (rc) return rc;
    if (dt_taken) {
        Control c;
        rc = read_ctl(h, &c);
        if (rc) return rc;
        *dt_taken = c.dt;
        return check_flags(c);
    }
    return ADERDG_OK;
}

int aderdg_advance(aderdg_t *h, double t_end, int64_t max_steps)
{
    if (!h) return fail(ADERDG_E_INVAL, "NULL handle");
    if (!std::isfinite(t_end) || max_steps < 0) return fail(ADERDG_E_INVAL, "bad t_end / max_steps");
    int rc = set_t_end(h, t_end);
    if (rc) return rc;
    constexpr int CHUNK = 16;
    if (!h->graph) {
        // capture CHUNK steps once; every replay re-reads dt and t on the device
        cudaStreamCaptureStatus st;
        bool ok = cudaStreamIsCapturing(h->stream, &st) == cudaSuccess && st == cudaStreamCaptureStatusNone &&
                  h->stream != nullptr;
        cudaGraph_t g = nullptr;
        if (ok && cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            for (int i = 0; i < CHUNK && ok; ++i) ok = enqueue_step(h) == ADERDG_OK;
            if (cudaStreamEndCapture(h->stream, &g) != cudaSuccess) ok = false;
            if (ok && cudaGraphInstantiate(&h->graph, g, 0) != cudaSuccess) { ok = false; h->graph = nullptr; }
            if (g) cudaGraphDestroy(g);
        }
        cudaGetLastError();  // a failed capture falls back to plain launches
        h->graph_steps = h->graph ? CHUNK : 0;
    }
    int64_t done = 0;
    while (done < max_steps) {
        const int64_t k = std::min<int64_t>(CHUNK, max_steps - done);
        if (h->graph && k == CHUNK) {
            CK(cudaGraphLaunch(h->graph, h->stream));
        } else {
            for (int64_t i = 0; i < k; ++i) {
                rc = enqueue_step(h);
                if (rc) return rc;
            }
        }
        done += k;
        Control c;
        rc = read_ctl(h, &c);
        if (rc) return rc;
        rc = check_flags(c);
        if (rc) return rc;
        if (!(c.t < t_end)) break;
    }
    return ADERDG_OK;
}

int aderdg_cfl_dt(aderdg_t *h, double *dt)
{
    if (!h || !dt) return fail(ADERDG_E_INVAL, "NULL argument");
    k_cfl_query<<<1, 32, 0, h->stream>>>(h->ctl, h->scratch + MASS_BLOCKS * 9);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(dt, h->scratch + MASS_BLOCKS * 9, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return ADERDG_OK;
}

int aderdg_mass(aderdg_t *h, double *per_var)
{
    if (!h || !per_var) return fail(ADERDG_E_INVAL, "NULL argument");
    double vol = 1.0;
    for (int d = 0; d < h->dim; ++d) vol *= h->dx[d];
    k_mass_partial<<<MASS_BLOCKS, MASS_THREADS, 0, h->stream>>>(h->u, h->E, h->NS, h->M, h->n, h->dim, h->basis, vol,
                                                                h->scratch);
    CK(cudaGetLastError());
    k_mass_final<<<1, 32, 0, h->stream>>>(h->scratch, MASS_BLOCKS, h->M, h->scratch + MASS_BLOCKS * 9 + 8);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(per_var, h->scratch + MASS_BLOCKS * 9 + 8, sizeof(double) * h->M, cudaMemcpyDeviceToHost,
                       h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return ADERDG_OK;
}

int aderdg_sync(aderdg_t *h)
{
    if (!h) return fail(ADERDG_E_INVAL, "NULL handle");
    Control c;
    int rc = read_ctl(h, &c);
    if (rc) return rc;
    return check_flags(c);
}

int aderdg_profile(aderdg_t *h, int enable)
{
    if (!h) return fail(ADERDG_E_INVAL, "NULL handle");
    if (enable && !h->ev[0])
        for (auto &e : h->ev) CK(cudaEventCreate(&e));
    if (h->graph) {  // a captured graph would keep the old recording choice
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
    h->profiling = enable != 0;
    return ADERDG_OK;
}

int aderdg_profile_read(aderdg_t *h, float *ms_predictor, float *ms_corrector)
{
    if (!h || !h->profiling) return fail(ADERDG_E_INVAL, "profiling is not enabled");
    CK(cudaEventSynchronize(h->ev[2]));
    float a = 0.f, b = 0.f;
    CK(cudaEventElapsedTime(&a, h->ev[0], h->ev[1]));
    CK(cudaEventElapsedTime(&b, h->ev[1], h->ev[2]));
    if (ms_predictor) *ms_predictor = a;
    if (ms_corrector) *ms_corrector = b;
    return ADERDG_OK;
}

}  // extern "C"
