// Tile-shape autotuner of the per-element kernels.
//
// The predictor and the corrector are compiled in NSHAPE_P / NSHAPE_C
// launch variants (CTA sizes; for the predictor also a second kernel
// layout) that compute the same results.  The tuner
// times every shape of one (PDE, d, N, precision) on a synthetic periodic
// mesh of about 2^21 nodes -- the cost of a step does not depend on the
// data, only on the shapes and sizes -- and keeps the fastest, per process
// and optionally in a text cache file (one line per key:
// "<key> <predictor shape> <corrector shape>").
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <utility>

#include <cuda_runtime.h>

#include "../../include/aderdg.h"
#include "basis.h"
#include "common.cuh"
#include "instances.h"
#include "tune.h"

namespace aderdg {
void set_last_error(const char *msg);

#define ADERDG_DECL(tag, D, NN)                   \
    const KernelSet *ks_##tag##D##d_n##NN##_f64(); \
    const KernelSet *ks_##tag##D##d_n##NN##_f32();
ADERDG_INSTANCES(ADERDG_DECL)
#undef ADERDG_DECL

#define ADERDG_CODE_advection ADERDG_PDE_ADVECTION
#define ADERDG_CODE_euler ADERDG_PDE_EULER
#define ADERDG_CODE_elastic ADERDG_PDE_ELASTICITY
#define ADERDG_CODE_diffuse ADERDG_PDE_DIFFUSE_ELASTICITY

const KernelSet *lookup_kernels(int pde, int dim, int N, int prec)
{
#define ADERDG_MATCH(tag, D, NN)                                       \
    if (pde == ADERDG_CODE_##tag && dim == D && N == NN)                  \
        return prec ? ks_##tag##D##d_n##NN##_f32() : ks_##tag##D##d_n##NN##_f64();
    ADERDG_INSTANCES(ADERDG_MATCH)
#undef ADERDG_MATCH
    return nullptr;
}

int limiter_kernels(int pde, int dim, int N, int prec, int guess, bool keep, LimKernels *out, const char **why)
{
    const KernelSet *k64 = lookup_kernels(pde, dim, N, ADERDG_FP64);
    const KernelSet *ks = lookup_kernels(pde, dim, N, prec);
    *why = nullptr;
    if (guess == ADERDG_GUESS_EXTRAP) {
        *why = "the subcell limiter needs a fresh predictor per step (no EXTRAP guess)";
        return ADERDG_E_UNSUPPORTED;
    }
    if (!ks || !k64 || !k64->lim_fv) {
        *why = "no subcell limiter for this (pde, dim, N): its shared memory does not fit";
        return ADERDG_E_UNSUPPORTED;
    }
    if (!ks->lim_couple) {  // both instances come from the same LimCfg: not expected to happen
        *why = "no coupling kernel compiled for this precision of the subcell limiter";
        return ADERDG_E_UNSUPPORTED;
    }
    // the FP32 path projects its subcell averages in FP32 (FP64 only for
    // decisions too close to call)
    const bool f32 = prec == ADERDG_MIXED_FP32;
    void (*minmax)(KParams) = keep ? (f32 ? k64->lim_minmax32_keep : k64->lim_minmax_keep)
                                   : (f32 ? k64->lim_minmax32 : k64->lim_minmax);
    *out = LimKernels{minmax, f32 ? k64->lim_detect32 : k64->lim_detect,
                      k64->lim_fv, ks->lim_couple, k64->lim_smem, f32 ? k64->lim_smem_w32 : k64->lim_smem_w,
                      f32 ? 32 : 1, k64->lim_init};
    const std::pair<void (*)(KParams), size_t> lk[5] = {{out->minmax, out->smem_w},
                                                        {out->detect, out->smem_w},
                                                        {out->fv, out->smem},
                                                        {out->couple, out->smem},
                                                        {out->init, out->smem}};
    for (const auto &k : lk)
        if (k.second > 48 * 1024 && cudaFuncSetAttribute((const void *)k.first, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                         (int)k.second) != cudaSuccess) {
            *why = "shared memory opt-in of the limiter failed";
            return ADERDG_E_CUDA;
        }
    return ADERDG_OK;
}
}  // namespace aderdg

using namespace aderdg;

namespace {

struct Choice {
    int pred, corr;
};

std::mutex g_mu;                        // guards g_table and the cache file
std::map<std::string, Choice> g_table;  // key -> shapes, this process

int fail(int code, const std::string &m)
{
    set_last_error(m.c_str());
    return code;
}

#define CKT(call)                                                                               \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess) {                                                                \
            rc = fail(ADERDG_E_CUDA, std::string(#call ": ") + cudaGetErrorString(e_));         \
            goto done;                                                                          \
        }                                                                                       \
    } while (0)

// "<pde> <dim> <N> <precision> <device name> <SM count>" (spaces in the
// device name replaced)
std::string make_key(int pde, int dim, int N, int prec)
{
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp p{};
    cudaGetDeviceProperties(&p, dev);
    std::string name = p.name;
    for (char &c : name)
        if (c == ' ' || c == '\t' || c == '\n') c = '_';
    char buf[256];
    std::snprintf(buf, sizeof(buf), "pde%d_d%d_N%d_p%d_%s_sm%d", pde, dim, N, prec, name.c_str(),
                  p.multiProcessorCount);
    return buf;
}

bool read_cache(const char *path, const std::string &key, Choice *out)
{
    if (!path) return false;
    FILE *f = std::fopen(path, "r");
    if (!f) return false;
    char k[256];
    int a = 0, b = 0;
    bool found = false;
    while (std::fscanf(f, "%255s %d %d", k, &a, &b) == 3) {
        if (key == k && a >= 0 && a < NSHAPE_P && b >= 0 && b < NSHAPE_C) {
            *out = {a, b};
            found = true;  // the last line for a key wins
        }
    }
    std::fclose(f);
    return found;
}

void append_cache(const char *path, const std::string &key, Choice c)
{
    if (!path) return;
    FILE *f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "%s %d %d\n", key.c_str(), c.pred, c.corr);
    std::fclose(f);
}

int opt_in(const TileShape &t)
{
    if (t.smem > 48 * 1024 &&
        cudaFuncSetAttribute((const void *)t.kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)t.smem) !=
            cudaSuccess)
        return fail(ADERDG_E_CUDA, "shared memory opt-in failed");
    return ADERDG_OK;
}

// Synthetic state: a valid background plus a small hashed perturbation
// (ideal gas: rho ~ 1, rho v ~ 0.1, rho E ~ 2.5, so p > 0; diffuse
// interface: alpha, lambda, mu, rho ~ 1).
__global__ void k_fill_synthetic(double *u, long long count, int M, int pde)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= count) return;
    unsigned long long h = (unsigned long long)i * 0x9E3779B97F4A7C15ull;
    h ^= h >> 29;
    h *= 0xBF58476D1CE4E5B9ull;
    h ^= h >> 32;
    const double r = double(h >> 11) * (1.0 / 9007199254740992.0);
    const int v = (int)(i % M);
    double base = 0.0;
    if (pde == ADERDG_PDE_EULER) base = v == 0 ? 1.0 : (v == M - 1 ? 2.5 : 0.1);
    if (pde == ADERDG_PDE_DIFFUSE_ELASTICITY && v >= M - 4) base = 1.0;
    u[i] = base + 0.01 * r;
}

// Milliseconds per launch of one shape (2 untimed launches, then the mean
// of 5).
int time_shape(const TileShape &t, KParams kp, long long E, cudaStream_t st, cudaEvent_t a, cudaEvent_t b,
               float *ms)
{
    int rc = opt_in(t);
    if (rc) return rc;
    kp.ntiles = (E + t.epb - 1) / t.epb;
    for (int i = 0; i < 7; ++i) {
        if (i == 2) cudaEventRecord(a, st);
        t.kernel<<<(unsigned)kp.ntiles, t.threads, t.smem, st>>>(kp);
    }
    cudaEventRecord(b, st);
    cudaError_t e = cudaEventSynchronize(b);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return fail(ADERDG_E_CUDA, std::string("autotune launch: ") + cudaGetErrorString(e));
    float total = 0.f;
    cudaEventElapsedTime(&total, a, b);
    *ms = total / 5.f;
    return ADERDG_OK;
}

// Times every shape of ks (m variables, PDE parameters pp) and returns the
// fastest; a shape within 2 % of the best keeps the lower index.
int measure(const KernelSet *ks, int pde, int dim, int N, int m, const PdeParams &pp, Choice *out, float *ms)
{
    int rc = ADERDG_OK;
    const int n = N + 1;
    const int NS = ipow(n, dim), NF = ipow(n, dim - 1), NREC = 2 * dim * NF;
    const long long target = std::max(1LL, (1LL << 21) / NS);
    const int k = std::max(2, (int)std::ceil(std::pow((double)target, 1.0 / dim) - 1e-9));
    long long E = 1;
    for (int d = 0; d < dim; ++d) E *= k;
    const size_t nstate = (size_t)E * NS * m;
    double *u = nullptr, *uo = nullptr, *ref = nullptr;
    void *V = nullptr, *tr = nullptr;
    Control *ctl = nullptr;
    SolveDesc *dd = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t ea = nullptr, eb = nullptr;
    KParams kp;
    SolveDesc sd;
    Control c;
    Choice best{0, 0};
    float bp = 0.f, bc = 0.f;

    std::memset(&kp, 0, sizeof(kp));
    std::memset(&sd, 0, sizeof(sd));
    std::memset(&c, 0, sizeof(c));
    CKT(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    CKT(cudaEventCreate(&ea));
    CKT(cudaEventCreate(&eb));
    CKT(cudaMalloc(&u, nstate * sizeof(double)));
    CKT(cudaMalloc(&uo, nstate * sizeof(double)));
    CKT(cudaMalloc(&V, nstate * ks->elem_bytes));
    CKT(cudaMalloc(&tr, (size_t)E * NREC * ks->rs * ks->elem_bytes));
    CKT(cudaMalloc(&ref, sizeof(double) * (size_t)E * (ks->rf > 0 ? ks->rf : 1)));
    CKT(cudaMalloc(&ctl, sizeof(Control)));
    CKT(cudaMalloc(&dd, sizeof(SolveDesc)));

    sd.E = E;
    for (int d = 0; d < 3; ++d) {
        sd.cells[d] = d < dim ? k : 1;
        sd.inv_dx[d] = d < dim ? (double)k : 1.0;  // unit box
    }
    fill_desc_spacing(sd);
    fill_desc_lift(sd, N);
    sd.picard = n;
    sd.u = u;
    sd.u_out = uo;
    sd.V = V;
    sd.tr = tr;
    sd.ref = ks->rf > 0 ? ref : nullptr;
    sd.ctl = ctl;
    c.dim = dim;
    c.alpha = default_alpha(N);
    for (int d = 0; d < 3; ++d) c.inv_dx[d] = sd.inv_dx[d];
    kp.solves = dd;
    kp.nsolves = 1;
    kp.use_ctl_dt = 0;
    kp.dt_arg = 1e-3 / k;
    kp.pde = pp;
    if (build_basis(N, kp.b)) {
        rc = fail(ADERDG_E_INVAL, "basis construction failed");
        goto done;
    }
    fill_ops(kp);
    k_fill_synthetic<<<(unsigned)((nstate + 255) / 256), 256, 0, st>>>(u, (long long)nstate, m, pde);
    CKT(cudaGetLastError());
    CKT(cudaMemcpyAsync(dd, &sd, sizeof(sd), cudaMemcpyHostToDevice, st));
    CKT(cudaMemcpyAsync(ctl, &c, sizeof(c), cudaMemcpyHostToDevice, st));

    for (int i = 0; i < NSHAPE_P; ++i) {
        float t = 0.f;
        if ((rc = time_shape(ks->pshape[i], kp, E, st, ea, eb, &t))) goto done;
        if (ms) ms[i] = t;
        if (i == 0 || t < 0.98f * bp) { best.pred = i; bp = t; }
    }
    for (int i = 0; i < NSHAPE_C; ++i) {
        float t = 0.f;
        if ((rc = time_shape(ks->cshape[i], kp, E, st, ea, eb, &t))) goto done;
        if (ms) ms[NSHAPE_P + i] = t;
        if (i == 0 || t < 0.98f * bc) { best.corr = i; bc = t; }
    }
    *out = best;
done:
    if (st) cudaStreamSynchronize(st);
    cudaFree(u);
    cudaFree(uo);
    cudaFree(V);
    cudaFree(tr);
    cudaFree(ref);
    cudaFree(ctl);
    cudaFree(dd);
    if (ea) cudaEventDestroy(ea);
    if (eb) cudaEventDestroy(eb);
    if (st) cudaStreamDestroy(st);
    return rc;
}

int nvar_of(int pde, int dim) { return pde_nvar(pde, dim); }

// Shapes for a key: process table, cache file, or a measurement.
int tuned(const KernelSet *ks, int pde, int dim, int N, int prec, const PdeParams &pp, const char *cache, bool force,
          Choice *out, float *ms)
{
    const std::string key = make_key(pde, dim, N, prec);
    std::lock_guard<std::mutex> lk(g_mu);
    if (ms)
        for (int i = 0; i < NSHAPE_P + NSHAPE_C; ++i) ms[i] = -1.f;
    if (!force) {
        auto it = g_table.find(key);
        if (it != g_table.end()) { *out = it->second; return ADERDG_OK; }
        if (read_cache(cache, key, out)) { g_table[key] = *out; return ADERDG_OK; }
    }
    Choice c{0, 0};
    const int rc = measure(ks, pde, dim, N, nvar_of(pde, dim), pp, &c, ms);
    if (rc) return rc;
    g_table[key] = c;
    append_cache(cache, key, c);
    *out = c;
    return ADERDG_OK;
}

}  // namespace

namespace aderdg {

int resolve_shapes(const KernelSet *ks, int pde, int dim, int N, int prec, const PdeParams &pp, int pred_req,
                   int corr_req, const char *cache, bool extrap, KernelSet *out)
{
    if (!valid_shape_requests(pred_req, corr_req)) return fail(ADERDG_E_INVAL, "bad tile shape request");
    Choice c{pred_req, corr_req};
    if (pred_req == ADERDG_SHAPE_AUTOTUNE || corr_req == ADERDG_SHAPE_AUTOTUNE) {
        Choice t{0, 0};
        const int rc = tuned(ks, pde, dim, N, prec, pp, cache, false, &t, nullptr);
        if (rc) return rc;
        if (pred_req == ADERDG_SHAPE_AUTOTUNE) c.pred = t.pred;
        if (corr_req == ADERDG_SHAPE_AUTOTUNE) c.corr = t.corr;
    }
    *out = with_shapes(*ks, c.pred, c.corr, extrap);
    int rc = opt_in(extrap ? ks->pshape_ex[c.pred] : ks->pshape[c.pred]);
    if (!rc) rc = opt_in(ks->cshape[c.corr]);
    return rc;
}

}  // namespace aderdg

extern "C" int aderdg_autotune(const aderdg_solve_spec_t *spec, int precision, const char *tune_cache, int flags,
                               int shapes[2], float *ms)
{
    if (!spec || !shapes) return fail(ADERDG_E_INVAL, "aderdg_autotune: spec/shapes is NULL");
    if (precision != ADERDG_FP64 && precision != ADERDG_MIXED_FP32) return fail(ADERDG_E_INVAL, "bad precision");
    const KernelSet *ks = lookup_kernels(spec->pde.kind, spec->mesh.dim, spec->N, precision);
    if (!ks) return fail(ADERDG_E_UNSUPPORTED, "no kernels compiled for this (pde, dim, N)");
    PdeParams pp;
    for (int i = 0; i < 8; ++i) pp.p[i] = spec->pde.p[i];
    fill_pde_consts(spec->pde.kind, pp);
    Choice c{0, 0};
    const int rc = tuned(ks, spec->pde.kind, spec->mesh.dim, spec->N, precision, pp, tune_cache,
                         (flags & ADERDG_TUNE_FORCE) != 0, &c, ms);
    if (rc) return rc;
    shapes[0] = c.pred;
    shapes[1] = c.corr;
    return ADERDG_OK;
}
