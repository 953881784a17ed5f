// aderdg_step_noalloc: one ADER-DG step (predictor + corrector, given dt)
// on caller-owned device buffers, with no device allocation at all.
//
// Who needs it: callers that cannot call cudaMalloc -- hosts whose device
// memory is owned by another allocator that must account for every byte,
// code paths where cudaMalloc's implicit device synchronisation is not
// acceptable, and embedded or real-time callers that forbid allocation
// after start-up.  The regular handle API allocates its volume-term and
// face-trace buffers at aderdg_create; this entry point keeps them in one
// fixed, file-scope device array instead.
//
// The scratch array below (ADERDG_NOALLOC_SCRATCH_BYTES = 32 MiB) is part
// of the module: every GPU that loads the library holds it until the
// process exits.  All calls share it and it keeps the last call's
// contents, so two calls whose work overlaps on the GPU (different streams,
// or different host threads) race on it; serialise them.
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include <cuda_runtime.h>

#include "../../include/aderdg.h"
#include "basis.h"
#include "common.cuh"
#include "tune.h"

namespace aderdg {
void set_last_error(const char *msg);
}  // namespace aderdg

using namespace aderdg;

namespace {

constexpr size_t SCRATCH_BYTES = ADERDG_NOALLOC_SCRATCH_BYTES;

// The scratch: volume term, face-trace records and the control block of
// the step in flight.  Host code must not pass this name to a kernel (on
// the host it is only a stand-in); it uses the device address that
// cudaGetSymbolAddress returns.
static __device__ __align__(256) unsigned char g_noalloc_scratch[SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
void *g_scratch_dev[MAX_DEVICES] = {};

int fail(int code, const std::string &m)
{
    set_last_error(m.c_str());
    return code;
}

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

const KernelSet *kernels_for(int pde, int dim, int N, int prec)
{
    return lookup_kernels(pde, dim, N, prec);
}

// Puts the step's descriptor into the scratch (it arrives by value as a
// kernel argument, so no host buffer has to outlive the call) and clears
// the control block: the corrector max-reduces wave speeds and ORs flags
// into it, so it must start at zero on every call.
static_assert(sizeof(Control) % sizeof(unsigned int) == 0, "control block is cleared word by word");
__global__ void k_noalloc_setup(const SolveDesc sd, SolveDesc *d_desc, Control *ctl)
{
    if (blockIdx.x != 0) return;
    if (threadIdx.x == 0) *d_desc = sd;
    unsigned int *c = reinterpret_cast<unsigned int *>(ctl);
    for (int i = threadIdx.x; i < (int)(sizeof(Control) / sizeof(unsigned int)); i += blockDim.x) c[i] = 0u;
}

// Device address of the scratch on the current device; looked up once per
// device (with that device current) and cached.
int scratch_address(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(ADERDG_E_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= MAX_DEVICES) return fail(ADERDG_E_CUDA, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_dev[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return fail(ADERDG_E_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
        g_scratch_dev[dev] = p;
    }
    *out = g_scratch_dev[dev];
    return ADERDG_OK;
}

}  // namespace

extern "C" int aderdg_step_noalloc(const aderdg_mesh_t *mesh, int N, int nVar, const aderdg_pde_t *pde,
                                   int precision, int picard_iters, const double *u_in, double *u_out,
                                   double dt, void *cuda_stream)
{
    if (!mesh || !pde || !u_in || !u_out) return fail(ADERDG_E_INVAL, "NULL argument");
    // the same mesh and parameter limits as aderdg_create (cells[d] <= 2^30,
    // E <= 2^31, PDE parameter ranges), before any size is computed from them
    long long E = 0;
    const char *why = nullptr;
    if (check_mesh(*mesh, pde->kind, &E, &why)) return fail(ADERDG_E_INVAL, why);
    const int m = pde_nvar(pde->kind, mesh->dim);
    if (nVar != m) return fail(ADERDG_E_INVAL, "nVar does not match the PDE");
    if (precision != ADERDG_FP64 && precision != ADERDG_MIXED_FP32) return fail(ADERDG_E_INVAL, "bad precision");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(ADERDG_E_INVAL, "dt must be positive and finite");
    const KernelSet *ks = (N >= 1 && N <= 9) ? kernels_for(pde->kind, mesh->dim, N, precision) : nullptr;
    if (!ks) return fail(ADERDG_E_UNSUPPORTED, "no kernels compiled for this (pde, dim, N)");
    if (check_pde_params(*pde, &why)) return fail(ADERDG_E_INVAL, why);
    const int n = N + 1;
    const int NS = ipow(n, mesh->dim), NF = ipow(n, mesh->dim - 1), NREC = mesh->dim * 2 * NF;
    const size_t v_bytes = align256((size_t)E * NS * m * ks->elem_bytes);
    const size_t tr_bytes = align256((size_t)E * NREC * ks->rs * ks->elem_bytes);
    const size_t ref_bytes = align256((size_t)E * ks->rf * sizeof(double));
    const size_t need = v_bytes + tr_bytes + align256(sizeof(Control)) + align256(sizeof(SolveDesc)) + ref_bytes;
    if (need > SCRATCH_BYTES)
        return fail(ADERDG_E_INVAL, "mesh too large for the static scratch: needs " + std::to_string(need) +
                                        " bytes, limit " + std::to_string(SCRATCH_BYTES) + " bytes");

    void *base = nullptr;
    int rc = scratch_address(&base);
    if (rc) return rc;
    unsigned char *sb = static_cast<unsigned char *>(base);
    Control *ctl = reinterpret_cast<Control *>(sb + v_bytes + tr_bytes);
    SolveDesc *d_desc = reinterpret_cast<SolveDesc *>(sb + v_bytes + tr_bytes + align256(sizeof(Control)));
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);

    SolveDesc sd;
    std::memset(&sd, 0, sizeof(sd));
    sd.E = E;
    for (int d = 0; d < 3; ++d) {
        sd.cells[d] = d < mesh->dim ? (int)mesh->cells[d] : 1;
        sd.inv_dx[d] = d < mesh->dim ? 1.0 / ((mesh->hi[d] - mesh->lo[d]) / mesh->cells[d]) : 1.0;
    }
    fill_desc_spacing(sd);
    fill_desc_lift(sd, N);
    sd.picard = picard_iters > 0 ? picard_iters : N + 1;
    sd.u = u_in;
    sd.u_out = u_out;
    sd.V = sb;
    sd.tr = sb + v_bytes;
    sd.ref = ks->rf > 0 ? reinterpret_cast<double *>(sb + v_bytes + tr_bytes + align256(sizeof(Control)) +
                                                     align256(sizeof(SolveDesc)))
                        : nullptr;
    sd.ctl = ctl;

    KParams kp;
    std::memset(&kp, 0, sizeof(kp));
    kp.solves = d_desc;
    kp.nsolves = 1;
    kp.dt_arg = dt;
    kp.use_ctl_dt = 0;
    for (int i = 0; i < 8; ++i) kp.pde.p[i] = pde->p[i];
    fill_pde_consts(pde->kind, kp.pde);
    if (build_basis(N, kp.b)) return fail(ADERDG_E_INVAL, "basis construction failed");
    fill_ops(kp);

    // large shared-memory kernels need the opt-in (no allocation involved)
    if (ks->pred_smem > 48 * 1024 &&
        cudaFuncSetAttribute((const void *)ks->predictor, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)ks->pred_smem) != cudaSuccess)
        return fail(ADERDG_E_CUDA, "predictor shared-memory opt-in failed");
    if (ks->corr_smem > 48 * 1024 &&
        cudaFuncSetAttribute((const void *)ks->corrector, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)ks->corr_smem) != cudaSuccess)
        return fail(ADERDG_E_CUDA, "corrector shared-memory opt-in failed");

    k_noalloc_setup<<<1, 32, 0, st>>>(sd, d_desc, ctl);
    kp.ntiles = (E + ks->pred_epb - 1) / ks->pred_epb;
    ks->predictor<<<(unsigned)kp.ntiles, ks->pred_threads, ks->pred_smem, st>>>(kp);
    kp.ntiles = (E + ks->corr_epb - 1) / ks->corr_epb;
    ks->corrector<<<(unsigned)kp.ntiles, ks->corr_threads, ks->corr_smem, st>>>(kp);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(ADERDG_E_CUDA, std::string("launch: ") + cudaGetErrorString(e));
    return ADERDG_OK;
}
