// Domain decomposition of one periodic Cartesian mesh into blocks, with the
// step structure of the paper's distributed-memory ADER-DG (Sec. 2.2, the
// closing remarks on MPI; Sec. 4, strong scaling): each block runs the
// predictor on its boundary elements first, sends the time-averaged face
// traces (qbar, Fbar_n, wave speed) of those elements to its neighbours
// while the predictor of its interior elements runs, and the corrector then
// reads the received traces across the block faces.  The time step needs
// one global reduction per step: a max-reduction of the per-direction wave
// speeds (dt = alpha / sum_d lambda_d^max / dx_d with the global maxima),
// which makes every block take the dt of the undivided mesh.
//
// Here all blocks live on one GPU: the "send" is a kernel that stores each
// block's boundary chunks into its neighbours' halo buffers, on a second
// stream that overlaps the interior predictor, and the reduction is a
// one-thread kernel over the blocks' control blocks.  Each block's
// arithmetic is the undivided mesh's arithmetic on the same data, so the
// result is bitwise that of the single-domain solver.
//
// The plan functions (aderdg_dd_plan, aderdg_dd_face_elements,
// aderdg_dd_element_lists) are plain host code: which block owns which
// cells, who neighbours whom, which elements send which chunk, in which
// order a receiver stores it.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/aderdg.h"
#include "basis.h"
#include "common.cuh"
#include "control.cuh"
#include "tune.h"

namespace aderdg {
void set_last_error(const char *msg);
}  // namespace aderdg

using namespace aderdg;

namespace {

int fail(int code, const std::string &m)
{
    set_last_error(m.c_str());
    return code;
}

#define CKD(call)                                                                                          \
    do {                                                                                                   \
        cudaError_t e_ = (call);                                                                           \
        if (e_ != cudaSuccess) return fail(ADERDG_E_CUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
    } while (0)

// ---------------------------------------------------------------------------
// the plan (host logic)
// ---------------------------------------------------------------------------

// Cells of block i of p blocks along a direction of C cells, and its first
// cell: the first C mod p blocks take one cell more.
void split1(long long C, int p, int i, long long *cells, long long *offset)
{
    const long long base = C / p, rem = C % p;
    *cells = base + (i < rem ? 1 : 0);
    *offset = i * base + std::min<long long>(i, rem);
}

int check_parts(const aderdg_mesh_t &m, const int *parts, int rank, long long *Eg)
{
    const char *why = nullptr;
    if (check_mesh(m, ADERDG_PDE_ADVECTION, Eg, &why)) return fail(ADERDG_E_INVAL, why);
    if (!parts) return fail(ADERDG_E_INVAL, "parts is NULL");
    long long K = 1;
    for (int d = 0; d < m.dim; ++d) {
        if (parts[d] < 1 || parts[d] > m.cells[d])
            return fail(ADERDG_E_INVAL, "parts[d] must be in 1 .. cells[d]");
        K *= parts[d];
    }
    if (K > 4096) return fail(ADERDG_E_INVAL, "at most 4096 blocks");
    if (rank < 0 || rank >= K) return fail(ADERDG_E_INVAL, "rank out of range");
    return ADERDG_OK;
}

// Block `rank` (x-fastest over the block grid) of the plan.
void plan_block(const aderdg_mesh_t &m, const int *parts, int rank, aderdg_dd_block_t *b)
{
    std::memset(b, 0, sizeof(*b));
    b->rank = rank;
    int r = rank;
    for (int d = 0; d < 3; ++d) {
        const int p = d < m.dim ? parts[d] : 1;
        b->coords[d] = r % p;
        r /= p;
    }
    b->elements = 1;
    b->boundary_elements = 0;
    for (int d = 0; d < 3; ++d) {
        long long c = 1, o = 0;
        if (d < m.dim) split1(m.cells[d], parts[d], b->coords[d], &c, &o);
        b->cells[d] = c;
        b->offset[d] = o;
        b->elements *= c;
    }
    for (int d = 0; d < 3; ++d)
        for (int side = 0; side < 2; ++side) {
            if (d >= m.dim || parts[d] == 1) {
                b->neighbour[d][side] = -1;
                b->face_chunks[d][side] = 0;
                continue;
            }
            int c[3] = {b->coords[0], b->coords[1], b->coords[2]};
            c[d] = (c[d] + (side ? 1 : parts[d] - 1)) % parts[d];
            const int px = parts[0], py = m.dim > 1 ? parts[1] : 1;
            b->neighbour[d][side] = c[0] + px * (c[1] + py * c[2]);
            b->face_chunks[d][side] = b->elements / b->cells[d];
        }
    // elements with a face on a split boundary
    long long inner = 1;
    for (int d = 0; d < 3; ++d) {
        const bool split = d < m.dim && parts[d] > 1;
        inner *= split ? std::max<long long>(0, b->cells[d] - 2) : b->cells[d];
    }
    b->boundary_elements = b->elements - inner;
}

// Block-local index of the element at position k along d and transverse
// index j (the other directions, lowest fastest).
long long face_element(const aderdg_dd_block_t &b, int d, long long k, long long j)
{
    long long ix, iy, iz;
    const long long cx = b.cells[0], cy = b.cells[1];
    if (d == 0) { ix = k; iy = j % cy; iz = j / cy; }
    else if (d == 1) { ix = j % cx; iy = k; iz = j / cx; }
    else { ix = j % cx; iy = j / cx; iz = k; }
    return ix + cx * (iy + cy * iz);
}

void element_lists(const aderdg_mesh_t &m, const int *parts, const aderdg_dd_block_t &b, std::vector<int> *bnd,
                   std::vector<int> *inn)
{
    bnd->clear();
    inn->clear();
    for (long long iz = 0; iz < b.cells[2]; ++iz)
        for (long long iy = 0; iy < b.cells[1]; ++iy)
            for (long long ix = 0; ix < b.cells[0]; ++ix) {
                const long long k[3] = {ix, iy, iz};
                bool edge = false;
                for (int d = 0; d < m.dim; ++d)
                    if (parts[d] > 1 && (k[d] == 0 || k[d] == b.cells[d] - 1)) edge = true;
                (edge ? bnd : inn)->push_back((int)(ix + b.cells[0] * (iy + b.cells[1] * iz)));
            }
}

}  // namespace

extern "C" int aderdg_dd_plan(const aderdg_mesh_t *mesh, const int parts[3], int rank, aderdg_dd_block_t *block)
{
    if (!mesh || !block) return fail(ADERDG_E_INVAL, "NULL argument");
    long long Eg = 0;
    const int rc = check_parts(*mesh, parts, rank, &Eg);
    if (rc) return rc;
    plan_block(*mesh, parts, rank, block);
    return ADERDG_OK;
}

extern "C" int aderdg_dd_face_elements(const aderdg_mesh_t *mesh, const int parts[3], int rank, int d, int side,
                                       int64_t *elements)
{
    if (!mesh || !elements) return fail(ADERDG_E_INVAL, "NULL argument");
    long long Eg = 0;
    const int rc = check_parts(*mesh, parts, rank, &Eg);
    if (rc) return rc;
    if (d < 0 || d >= mesh->dim || (side != 0 && side != 1)) return fail(ADERDG_E_INVAL, "bad face");
    aderdg_dd_block_t b;
    plan_block(*mesh, parts, rank, &b);
    const long long cnt = b.elements / b.cells[d];
    for (long long j = 0; j < cnt; ++j) elements[j] = face_element(b, d, side ? b.cells[d] - 1 : 0, j);
    return ADERDG_OK;
}

extern "C" int aderdg_dd_element_lists(const aderdg_mesh_t *mesh, const int parts[3], int rank, int64_t *boundary,
                                       int64_t *interior)
{
    if (!mesh) return fail(ADERDG_E_INVAL, "NULL argument");
    long long Eg = 0;
    const int rc = check_parts(*mesh, parts, rank, &Eg);
    if (rc) return rc;
    aderdg_dd_block_t b;
    plan_block(*mesh, parts, rank, &b);
    std::vector<int> bl, il;
    element_lists(*mesh, parts, b, &bl, &il);
    if (boundary) std::copy(bl.begin(), bl.end(), boundary);
    if (interior) std::copy(il.begin(), il.end(), interior);
    return ADERDG_OK;
}

// ---------------------------------------------------------------------------
// the partitioned solver (all blocks on the current GPU)
// ---------------------------------------------------------------------------

namespace {

// One face of one block whose boundary chunks go to a neighbour's halo:
// the chunks (d, side) of the elements at position k = side ? c_d - 1 : 0
// along d, in transverse order j, and their reference states.
struct ExJob {
    const unsigned long long *src;  // the block's traces, 8-byte words
    const double *src_ref;          // its reference states (FP32 path) or NULL
    unsigned long long *dst;        // the neighbour's halo_tr[d][1 - side]
    double *dst_ref;                // the neighbour's halo_ref[d][1 - side] or NULL
    long long cells[3];
    long long count;                // chunks (elements on the face)
    int dim, d, side;
};

struct Block {
    aderdg_dd_block_t plan{};
    long long E = 0;
    double *u = nullptr;
    void *V = nullptr, *tr = nullptr, *qprev = nullptr;
    double *ref = nullptr;
    Control *ctl = nullptr;
    void *halo_tr[3][2] = {};
    double *halo_ref[3][2] = {};
    int *blist = nullptr, *ilist = nullptr;
    long long nb = 0, ni = 0;
};

// The global time step: the per-direction wave-speed maxima of every block
// (bit patterns of non-negative doubles: integer max == double max, order
// free), a non-finite flag raised anywhere stops every block, then each
// block's CFL step from the common maxima (the same dt and t everywhere).
__global__ void k_dt_dd(Control *const *ctls, int K)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    unsigned long long lam[3] = {0ull, 0ull, 0ull};
    unsigned int bad = 0u;
    for (int k = 0; k < K; ++k) {
        for (int d = 0; d < 3; ++d) lam[d] = ctls[k]->lam_acc[d] > lam[d] ? ctls[k]->lam_acc[d] : lam[d];
        bad |= ctls[k]->flags & FLAG_NONFINITE;
    }
    for (int k = 0; k < K; ++k) {
        Control *c = ctls[k];
        for (int d = 0; d < 3; ++d) c->lam_acc[d] = lam[d];
        c->flags |= bad;
        dt_update(c);
    }
}

// The exchange: the face chunks of every job, in 8-byte words, stored into
// the neighbours' halos, then the reference states (FP32 path) of the same
// elements.  blockIdx.y = job.
__global__ void k_dd_exchange(const ExJob *jobs, int njobs, int words, int rf)
{
    if ((int)blockIdx.y >= njobs) return;
    const ExJob &J = jobs[blockIdx.y];
    const long long nt = J.count * words;
    const long long total = nt + (J.dst_ref ? J.count * rf : 0);
    const long long cx = J.cells[0], cy = J.cells[1], cd = J.cells[J.d];
    const long long k = J.side ? cd - 1 : 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const bool tr = i < nt;
        const long long per = tr ? words : rf;
        const long long ii = tr ? i : i - nt;
        const long long j = ii / per, w = ii - j * per;
        long long ix, iy, iz;
        if (J.d == 0) { ix = k; iy = j % cy; iz = j / cy; }
        else if (J.d == 1) { ix = j % cx; iy = k; iz = j / cx; }
        else { ix = j % cx; iy = j / cx; iz = k; }
        const long long e = ix + cx * (iy + cy * iz);
        if (tr) J.dst[j * words + w] = J.src[((e * J.dim + J.d) * 2 + J.side) * words + w];
        else J.dst_ref[j * rf + w] = J.src_ref[e * rf + w];
    }
}

}  // namespace

struct aderdg_dd_s {
    int dim = 0, N = 0, n = 0, M = 0, pde = 0, precision = 0, picard = 0, guess = 0, K = 0;
    int parts[3] = {1, 1, 1};
    long long cells[3] = {1, 1, 1};
    long long Eg = 0;
    int NS = 0, NF = 0, NREC = 0;
    double alpha = 0, inv_dx[3] = {1, 1, 1};
    KernelSet kso{};
    cudaStream_t stream = nullptr, side = nullptr;
    bool own_stream = false;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    aderdg_alloc_t alloc{};
    bool has_alloc = false;
    size_t device_bytes = 0;
    std::vector<Block> blocks;
    SolveDesc *d_desc = nullptr;  // [3K]: boundary lists, interior lists, whole blocks
    long long ntiles_b = 0, ntiles_i = 0, ntiles_c = 0;
    ExJob *d_jobs = nullptr;
    int njobs = 0, words = 0;
    long long max_chunks = 0;
    size_t halo_bytes = 0;  // per step
    Control **d_ctls = nullptr;
    Control *host_ctl = nullptr;  // pinned, K entries
    KParams kp{};
    cudaGraphExec_t graph = nullptr;
};

namespace {

void *dd_alloc(aderdg_dd_t *h, size_t bytes)
{
    void *p = nullptr;
    bytes = (bytes + 255) / 256 * 256;
    if (h->has_alloc) p = h->alloc.alloc(bytes, h->alloc.ctx);
    else if (cudaMalloc(&p, bytes) != cudaSuccess) { cudaGetLastError(); p = nullptr; }
    if (p) h->device_bytes += bytes;
    return p;
}

void dd_free(aderdg_dd_t *h, void *p)
{
    if (!p) return;
    if (h->has_alloc) h->alloc.free(p, h->alloc.ctx);
    else cudaFree(p);
}

__global__ void k_dd_set_t_end(Control *const *ctls, int K, double t_end)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < K) ctls[k]->t_end = t_end;
}

int dd_enqueue_step(aderdg_dd_t *h)
{
    const KernelSet *ks = &h->kso;
    KParams kp = h->kp;
    kp.use_ctl_dt = 1;
    k_dt_dd<<<1, 32, 0, h->stream>>>(h->d_ctls, h->K);
    CKD(cudaGetLastError());
    const bool exchange = h->njobs > 0 && h->ntiles_b > 0;
    if (h->ntiles_b > 0) {  // boundary elements first: their traces are sent
        kp.solves = h->d_desc;
        kp.nsolves = h->K;
        kp.ntiles = h->ntiles_b;
        ks->predictor<<<(unsigned)kp.ntiles, ks->pred_threads, ks->pred_smem, h->stream>>>(kp);
        CKD(cudaGetLastError());
    }
    if (exchange) {  // ... while the interior predictor runs
        CKD(cudaEventRecord(h->ev_fork, h->stream));
        CKD(cudaStreamWaitEvent(h->side, h->ev_fork, 0));
        const unsigned gx = (unsigned)std::max<long long>(1, std::min<long long>(64, (h->max_chunks * h->words + 255) / 256));
        k_dd_exchange<<<dim3(gx, (unsigned)h->njobs), 256, 0, h->side>>>(h->d_jobs, h->njobs, h->words, ks->rf);
        CKD(cudaGetLastError());
        CKD(cudaEventRecord(h->ev_join, h->side));
    }
    if (h->ntiles_i > 0) {
        kp.solves = h->d_desc + h->K;
        kp.nsolves = h->K;
        kp.ntiles = h->ntiles_i;
        ks->predictor<<<(unsigned)kp.ntiles, ks->pred_threads, ks->pred_smem, h->stream>>>(kp);
        CKD(cudaGetLastError());
    }
    if (exchange) CKD(cudaStreamWaitEvent(h->stream, h->ev_join, 0));
    kp.solves = h->d_desc + 2 * h->K;
    kp.nsolves = h->K;
    kp.ntiles = h->ntiles_c;
    ks->corrector<<<(unsigned)kp.ntiles, ks->corr_threads, ks->corr_smem, h->stream>>>(kp);
    CKD(cudaGetLastError());
    return ADERDG_OK;
}

int dd_read_ctls(aderdg_dd_t *h)
{
    for (int k = 0; k < h->K; ++k)
        CKD(cudaMemcpyAsync(h->host_ctl + k, h->blocks[k].ctl, sizeof(Control), cudaMemcpyDeviceToHost, h->stream));
    CKD(cudaStreamSynchronize(h->stream));
    return ADERDG_OK;
}

int dd_check_flags(const aderdg_dd_t *h)
{
    for (int k = 0; k < h->K; ++k) {
        if (h->host_ctl[k].flags & FLAG_NONFINITE) return fail(ADERDG_E_NONFINITE, "non-finite value in the state");
        if (h->host_ctl[k].flags & FLAG_TIMEOUT) return fail(ADERDG_E_TIMEOUT, "bounded device wait expired");
    }
    return ADERDG_OK;
}

int dd_set_t_end(aderdg_dd_t *h, double t_end)
{
    k_dd_set_t_end<<<(h->K + 127) / 128, 128, 0, h->stream>>>(h->d_ctls, h->K, t_end);
    CKD(cudaGetLastError());
    return ADERDG_OK;
}

// Copies between the global state (x-fastest elements) and block k's
// state: one 2D copy per z-slice of the block (rows of cx elements are
// contiguous in both).
int dd_copy_block(aderdg_dd_t *h, int k, double *global, bool to_block, cudaMemcpyKind kind)
{
    const Block &b = h->blocks[k];
    const size_t node = (size_t)h->NS * h->M * sizeof(double);
    const size_t gpitch = (size_t)h->cells[0] * node, bpitch = (size_t)b.plan.cells[0] * node;
    for (long long lz = 0; lz < b.plan.cells[2]; ++lz) {
        const long long gz = b.plan.offset[2] + lz;
        char *g = reinterpret_cast<char *>(global) +
                  ((size_t)(gz * h->cells[1] + b.plan.offset[1]) * h->cells[0] + b.plan.offset[0]) * node;
        char *l = reinterpret_cast<char *>(b.u) + (size_t)lz * b.plan.cells[1] * bpitch;
        if (to_block) CKD(cudaMemcpy2DAsync(l, bpitch, g, gpitch, bpitch, b.plan.cells[1], kind, h->stream));
        else CKD(cudaMemcpy2DAsync(g, gpitch, l, bpitch, bpitch, b.plan.cells[1], kind, h->stream));
    }
    return ADERDG_OK;
}

}  // namespace

extern "C" int aderdg_dd_destroy(aderdg_dd_t *h)
{
    if (!h) return ADERDG_OK;
    if (h->stream) cudaStreamSynchronize(h->stream);
    if (h->side) cudaStreamSynchronize(h->side);
    if (h->graph) cudaGraphExecDestroy(h->graph);
    for (Block &b : h->blocks) {
        dd_free(h, b.u);
        dd_free(h, b.V);
        dd_free(h, b.tr);
        dd_free(h, b.ref);
        dd_free(h, b.qprev);
        dd_free(h, b.ctl);
        dd_free(h, b.blist);
        dd_free(h, b.ilist);
        for (int d = 0; d < 3; ++d)
            for (int s = 0; s < 2; ++s) {
                dd_free(h, b.halo_tr[d][s]);
                dd_free(h, b.halo_ref[d][s]);
            }
    }
    dd_free(h, h->d_desc);
    dd_free(h, h->d_jobs);
    dd_free(h, h->d_ctls);
    if (h->host_ctl) cudaFreeHost(h->host_ctl);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    if (h->side) cudaStreamDestroy(h->side);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
    return ADERDG_OK;
}

extern "C" int aderdg_dd_create(const aderdg_mesh_t *mesh, int N, int nVar, const aderdg_pde_t *pde,
                                const aderdg_config_t *cfg, const int parts[3], aderdg_dd_t **out)
{
    if (!out) return fail(ADERDG_E_INVAL, "out is NULL");
    *out = nullptr;
    if (!mesh || !pde) return fail(ADERDG_E_INVAL, "mesh/pde is NULL");
    long long Eg = 0;
    const char *why = nullptr;
    if (check_mesh(*mesh, pde->kind, &Eg, &why)) return fail(ADERDG_E_INVAL, why);
    int rc = check_parts(*mesh, parts, 0, &Eg);
    if (rc) return rc;
    const int m = pde_nvar(pde->kind, mesh->dim);
    if (nVar != m) return fail(ADERDG_E_INVAL, "nVar does not match the PDE");
    if (N < 1 || N > 9) return fail(ADERDG_E_INVAL, "N must be in 1..9");
    const int prec = cfg ? cfg->precision : ADERDG_FP64;
    if (prec != ADERDG_FP64 && prec != ADERDG_MIXED_FP32) return fail(ADERDG_E_INVAL, "bad precision");
    const KernelSet *ks = lookup_kernels(pde->kind, mesh->dim, N, prec);
    if (!ks) return fail(ADERDG_E_UNSUPPORTED, "no kernels compiled for this (pde, dim, N)");
    if (check_pde_params(*pde, &why)) return fail(ADERDG_E_INVAL, why);
    const int guess = cfg ? cfg->initial_guess : ADERDG_GUESS_TRIVIAL;
    if (guess < ADERDG_GUESS_TRIVIAL || guess > ADERDG_GUESS_CERK) return fail(ADERDG_E_INVAL, "bad initial guess");
    if (cfg && cfg->limiter)
        return fail(ADERDG_E_UNSUPPORTED, "the subcell limiter is not available on a partitioned mesh");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return fail(ADERDG_E_CUDA, "no CUDA device available (the library has no CPU path)");
    }

    aderdg_dd_t *h = new aderdg_dd_s();
    h->dim = mesh->dim;
    h->N = N;
    h->n = N + 1;
    h->M = m;
    h->pde = pde->kind;
    h->precision = prec;
    h->guess = guess;
    h->picard = (cfg && cfg->picard_iters > 0) ? cfg->picard_iters : default_picard(N, guess);
    h->alpha = (cfg && cfg->cfl_alpha > 0) ? cfg->cfl_alpha : default_alpha(N);
    h->Eg = Eg;
    h->NS = ipow(h->n, h->dim);
    h->NF = ipow(h->n, h->dim - 1);
    h->NREC = h->dim * 2 * h->NF;
    h->K = 1;
    for (int d = 0; d < 3; ++d) {
        h->parts[d] = d < h->dim ? parts[d] : 1;
        h->cells[d] = d < h->dim ? mesh->cells[d] : 1;
        h->inv_dx[d] = d < h->dim ? 1.0 / ((mesh->hi[d] - mesh->lo[d]) / mesh->cells[d]) : 1.0;
        h->K *= h->parts[d];
    }
    PdeParams pp;
    for (int i = 0; i < 8; ++i) pp.p[i] = pde->p[i];
    fill_pde_consts(pde->kind, pp);
    rc = resolve_shapes(ks, pde->kind, h->dim, N, prec, pp, cfg ? cfg->pred_shape : 0, cfg ? cfg->corr_shape : 0,
                        cfg ? cfg->tune_cache : nullptr,
                        guess == ADERDG_GUESS_EXTRAP || guess == ADERDG_GUESS_CERK, &h->kso);
    if (rc) { delete h; return rc; }
    ks = &h->kso;
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
    if (cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming) != cudaSuccess) {
        aderdg_dd_destroy(h);
        return fail(ADERDG_E_CUDA, "stream / event creation failed");
    }
    KParams &kp = h->kp;
    std::memset(&kp, 0, sizeof(kp));
    for (int i = 0; i < 8; ++i) kp.pde.p[i] = pde->p[i];
    fill_pde_consts(pde->kind, kp.pde);
    if (build_basis(N, kp.b)) { aderdg_dd_destroy(h); return fail(ADERDG_E_INVAL, "basis construction failed"); }
    fill_ops(kp);
    h->words = (int)((size_t)h->NF * ks->rs * ks->elem_bytes / 8);

    // blocks: plan, element lists, buffers
    h->blocks.resize(h->K);
    bool ok = true;
    std::vector<std::vector<int>> bl(h->K), il(h->K);
    for (int k = 0; k < h->K && ok; ++k) {
        Block &b = h->blocks[k];
        plan_block(*mesh, h->parts, k, &b.plan);
        b.E = b.plan.elements;
        element_lists(*mesh, h->parts, b.plan, &bl[k], &il[k]);
        b.nb = (long long)bl[k].size();
        b.ni = (long long)il[k].size();
        const size_t nstate = (size_t)b.E * h->NS * m;
        b.u = (double *)dd_alloc(h, nstate * sizeof(double));
        b.V = dd_alloc(h, nstate * ks->elem_bytes);
        b.tr = dd_alloc(h, (size_t)b.E * h->NREC * ks->rs * ks->elem_bytes);
        b.ctl = (Control *)dd_alloc(h, sizeof(Control));
        ok = b.u && b.V && b.tr && b.ctl;
        if (ks->rf > 0) ok = ok && (b.ref = (double *)dd_alloc(h, sizeof(double) * (size_t)b.E * ks->rf));
        if (guess == ADERDG_GUESS_EXTRAP) ok = ok && (b.qprev = dd_alloc(h, nstate * h->n * ks->elem_bytes));
        if (b.nb > 0) ok = ok && (b.blist = (int *)dd_alloc(h, sizeof(int) * b.nb));
        if (b.ni > 0) ok = ok && (b.ilist = (int *)dd_alloc(h, sizeof(int) * b.ni));
        for (int d = 0; d < h->dim && ok; ++d)
            for (int s = 0; s < 2 && ok; ++s) {
                const long long cnt = b.plan.face_chunks[d][s];
                if (cnt == 0) continue;
                b.halo_tr[d][s] = dd_alloc(h, (size_t)cnt * h->words * 8);
                ok = b.halo_tr[d][s] != nullptr;
                if (ks->rf > 0) ok = ok && (b.halo_ref[d][s] = (double *)dd_alloc(h, sizeof(double) * cnt * ks->rf));
                h->max_chunks = std::max(h->max_chunks, cnt);
                h->halo_bytes += (size_t)cnt * ((size_t)h->words * 8 + (size_t)ks->rf * 8);
            }
    }
    h->d_desc = ok ? (SolveDesc *)dd_alloc(h, sizeof(SolveDesc) * 3 * h->K) : nullptr;
    h->d_ctls = ok ? (Control **)dd_alloc(h, sizeof(Control *) * h->K) : nullptr;
    if (!ok || !h->d_desc || !h->d_ctls) {
        aderdg_dd_destroy(h);
        return fail(ADERDG_E_NOMEM, "device allocation failed");
    }
    if (cudaMallocHost(&h->host_ctl, sizeof(Control) * h->K) != cudaSuccess) {
        h->host_ctl = nullptr;
        aderdg_dd_destroy(h);
        return fail(ADERDG_E_NOMEM, "pinned host allocation failed");
    }

    // descriptors: [0, K) boundary elements, [K, 2K) interior ones (both
    // predictor launches), [2K, 3K) whole blocks with their halos (corrector)
    std::vector<SolveDesc> sd(3 * h->K);
    std::vector<ExJob> jobs;
    std::vector<Control *> ctls(h->K);
    long long tb = 0, ti = 0, tc = 0;
    for (int k = 0; k < h->K; ++k) {
        Block &b = h->blocks[k];
        SolveDesc base;
        std::memset(&base, 0, sizeof(base));
        for (int d = 0; d < 3; ++d) {
            base.cells[d] = (int)b.plan.cells[d];
            base.inv_dx[d] = h->inv_dx[d];
        }
        fill_desc_spacing(base);
        fill_desc_lift(base, N);
        base.picard = h->picard;
        base.guess = h->guess;
        base.picard_first = default_picard(N, ADERDG_GUESS_ORDER3);
        base.u = b.u;
        base.u_out = b.u;
        base.V = b.V;
        base.tr = b.tr;
        base.ref = b.ref;
        base.qprev = b.qprev;
        base.ctl = b.ctl;
        SolveDesc &db = sd[k], &di = sd[h->K + k], &dc = sd[2 * h->K + k];
        db = base;
        db.E = b.nb;
        db.elist = b.blist;
        db.tile0_p = tb;
        tb += (b.nb + ks->pred_epb - 1) / ks->pred_epb;
        di = base;
        di.E = b.ni;
        di.elist = b.ilist;
        di.tile0_p = ti;
        ti += (b.ni + ks->pred_epb - 1) / ks->pred_epb;
        dc = base;
        dc.E = b.E;
        dc.tile0_c = tc;
        tc += (b.E + ks->corr_epb - 1) / ks->corr_epb;
        for (int d = 0; d < 3; ++d)
            for (int s = 0; s < 2; ++s) {
                dc.halo_tr[d][s] = b.halo_tr[d][s];
                dc.halo_ref[d][s] = b.halo_ref[d][s];
            }
        ctls[k] = b.ctl;
        // the chunks this block sends across each split face
        for (int d = 0; d < h->dim; ++d)
            for (int s = 0; s < 2; ++s) {
                const int nbk = b.plan.neighbour[d][s];
                if (nbk < 0) continue;
                ExJob J;
                std::memset(&J, 0, sizeof(J));
                J.src = reinterpret_cast<const unsigned long long *>(b.tr);
                J.src_ref = b.ref;
                J.dst = reinterpret_cast<unsigned long long *>(h->blocks[nbk].halo_tr[d][1 - s]);
                J.dst_ref = h->blocks[nbk].halo_ref[d][1 - s];
                for (int q = 0; q < 3; ++q) J.cells[q] = b.plan.cells[q];
                J.count = b.plan.face_chunks[d][s];
                J.dim = h->dim;
                J.d = d;
                J.side = s;
                jobs.push_back(J);
            }
    }
    h->ntiles_b = tb;
    h->ntiles_i = ti;
    h->ntiles_c = tc;
    h->njobs = (int)jobs.size();
    if (h->njobs > 65535) { aderdg_dd_destroy(h); return fail(ADERDG_E_INVAL, "too many block faces"); }
    if (h->njobs > 0 && !(h->d_jobs = (ExJob *)dd_alloc(h, sizeof(ExJob) * jobs.size()))) {
        aderdg_dd_destroy(h);
        return fail(ADERDG_E_NOMEM, "device allocation failed");
    }
    bool good = cudaMemcpyAsync(h->d_desc, sd.data(), sizeof(SolveDesc) * sd.size(), cudaMemcpyHostToDevice,
                                h->stream) == cudaSuccess &&
                cudaMemcpyAsync(h->d_ctls, ctls.data(), sizeof(Control *) * ctls.size(), cudaMemcpyHostToDevice,
                                h->stream) == cudaSuccess &&
                (h->njobs == 0 || cudaMemcpyAsync(h->d_jobs, jobs.data(), sizeof(ExJob) * jobs.size(),
                                                  cudaMemcpyHostToDevice, h->stream) == cudaSuccess);
    for (int k = 0; k < h->K && good; ++k) {
        Block &b = h->blocks[k];
        if (b.nb > 0)
            good = cudaMemcpyAsync(b.blist, bl[k].data(), sizeof(int) * b.nb, cudaMemcpyHostToDevice, h->stream) ==
                   cudaSuccess;
        if (good && b.ni > 0)
            good = cudaMemcpyAsync(b.ilist, il[k].data(), sizeof(int) * b.ni, cudaMemcpyHostToDevice, h->stream) ==
                   cudaSuccess;
        Control c;
        std::memset(&c, 0, sizeof(c));
        c.alpha = h->alpha;
        c.dim = h->dim;
        for (int d = 0; d < 3; ++d) c.inv_dx[d] = h->inv_dx[d];
        h->host_ctl[k] = c;
        good = good &&
               cudaMemcpyAsync(b.ctl, h->host_ctl + k, sizeof(Control), cudaMemcpyHostToDevice, h->stream) ==
                   cudaSuccess &&
               cudaMemsetAsync(b.u, 0, (size_t)b.E * h->NS * m * sizeof(double), h->stream) == cudaSuccess;
    }
    // the host copies (stack vectors, pinned staging) must outlive the copies
    good = good && cudaStreamSynchronize(h->stream) == cudaSuccess;
    if (!good) {
        aderdg_dd_destroy(h);
        return fail(ADERDG_E_CUDA, "initialisation failed");
    }
    *out = h;
    return ADERDG_OK;
}

extern "C" int aderdg_dd_set_state(aderdg_dd_t *h, const double *u, int where, double t)
{
    if (!h || !u) return fail(ADERDG_E_INVAL, "NULL argument");
    if (!std::isfinite(t)) return fail(ADERDG_E_INVAL, "t must be finite");
    const cudaMemcpyKind kind = where == ADERDG_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    for (int k = 0; k < h->K; ++k) {
        int rc = dd_copy_block(h, k, const_cast<double *>(u), true, kind);
        if (rc) return rc;
        Control c;
        std::memset(&c, 0, sizeof(c));
        c.t = t;
        c.t_end = t;
        c.alpha = h->alpha;
        c.dim = h->dim;
        for (int d = 0; d < 3; ++d) c.inv_dx[d] = h->inv_dx[d];
        h->host_ctl[k] = c;
        CKD(cudaMemcpyAsync(h->blocks[k].ctl, h->host_ctl + k, sizeof(Control), cudaMemcpyHostToDevice, h->stream));
        // wave-speed maxima of the block's state (combined over blocks by the next step)
        KParams kp = h->kp;
        kp.solves = h->d_desc + 2 * h->K + k;
        kp.nsolves = 1;
        const long long nodes = h->blocks[k].E * h->NS;
        h->kso.cfl<<<(unsigned)std::min<long long>(4 * 152, (nodes + 255) / 256), 256, 0, h->stream>>>(kp);
        CKD(cudaGetLastError());
    }
    CKD(cudaStreamSynchronize(h->stream));  // pageable source and the pinned staging
    return ADERDG_OK;
}

extern "C" int aderdg_dd_get_state(aderdg_dd_t *h, double *u, int where, double *t, int64_t *step)
{
    if (!h || !u) return fail(ADERDG_E_INVAL, "NULL argument");
    const cudaMemcpyKind kind = where == ADERDG_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    for (int k = 0; k < h->K; ++k) {
        const int rc = dd_copy_block(h, k, u, false, kind);
        if (rc) return rc;
    }
    int rc = dd_read_ctls(h);
    if (rc) return rc;
    if (t) *t = h->host_ctl[0].t;
    if (step) *step = h->host_ctl[0].step;
    return dd_check_flags(h);
}

extern "C" int aderdg_dd_step(aderdg_dd_t *h, double t_end, double *dt_taken)
{
    if (!h) return fail(ADERDG_E_INVAL, "NULL handle");
    if (!std::isfinite(t_end)) return fail(ADERDG_E_INVAL, "t_end must be finite");
    int rc = dd_set_t_end(h, t_end);
    if (rc) return rc;
    rc = dd_enqueue_step(h);
    if (rc) return rc;
    if (dt_taken) {
        rc = dd_read_ctls(h);
        if (rc) return rc;
        *dt_taken = h->host_ctl[0].dt;
        return dd_check_flags(h);
    }
    return ADERDG_OK;
}

extern "C" int aderdg_dd_advance(aderdg_dd_t *h, double t_end, int64_t max_steps)
{
    if (!h) return fail(ADERDG_E_INVAL, "NULL handle");
    if (!std::isfinite(t_end) || max_steps < 0) return fail(ADERDG_E_INVAL, "bad t_end / max_steps");
    int rc = dd_set_t_end(h, t_end);
    if (rc) return rc;
    constexpr int CHUNK = 16;
    if (!h->graph) {
        // CHUNK steps captured once (both streams: the exchange forks off and
        // joins back); every replay re-reads dt and t on the device
        cudaStreamCaptureStatus st;
        bool ok = cudaStreamIsCapturing(h->stream, &st) == cudaSuccess && st == cudaStreamCaptureStatusNone;
        cudaGraph_t g = nullptr;
        if (ok && cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            for (int i = 0; i < CHUNK && ok; ++i) ok = dd_enqueue_step(h) == ADERDG_OK;
            if (cudaStreamEndCapture(h->stream, &g) != cudaSuccess) ok = false;
            if (ok && cudaGraphInstantiate(&h->graph, g, 0) != cudaSuccess) { ok = false; h->graph = nullptr; }
            if (g) cudaGraphDestroy(g);
        }
        cudaGetLastError();  // a failed capture falls back to plain launches
    }
    int64_t done = 0;
    while (done < max_steps) {
        const int64_t k = std::min<int64_t>(CHUNK, max_steps - done);
        if (h->graph && k == CHUNK) {
            CKD(cudaGraphLaunch(h->graph, h->stream));
        } else {
            for (int64_t i = 0; i < k; ++i) {
                rc = dd_enqueue_step(h);
                if (rc) return rc;
            }
        }
        done += k;
        rc = dd_read_ctls(h);
        if (rc) return rc;
        rc = dd_check_flags(h);
        if (rc) return rc;
        if (!(h->host_ctl[0].t < t_end)) break;
    }
    return ADERDG_OK;
}

extern "C" int aderdg_dd_info(const aderdg_dd_t *h, int *blocks, int64_t *boundary_elements,
                              size_t *halo_bytes_per_step, size_t *device_bytes)
{
    if (!h) return fail(ADERDG_E_INVAL, "NULL handle");
    long long nb = 0;
    for (const Block &b : h->blocks) nb += b.nb;
    if (blocks) *blocks = h->K;
    if (boundary_elements) *boundary_elements = nb;
    if (halo_bytes_per_step) *halo_bytes_per_step = h->halo_bytes;
    if (device_bytes) *device_bytes = h->device_bytes;
    return ADERDG_OK;
}
