// Batched solves and the serving loop.
//
// Engine: a set of resident solves ("slots").  Slots are grouped by (PDE,
// dimension, degree, PDE parameters); every group gets one SolveDesc array
// in device memory, so a step is one dt kernel over all slots plus one
// predictor and one corrector launch per group, whatever the number of
// solves.  Membership can change between steps (continuous batching): the
// group arrays are rebuilt and the captured step graph is dropped.
//
// aderdg_batch_*   a fixed set of solves (one Engine, graph-replayed steps)
// aderdg_server_*  a request queue, device-memory admission and a
//                  background scheduler thread driving one Engine
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
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

#define CKB(call)                                                                          \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) return fail(ADERDG_E_CUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
    } while (0)

size_t a256(size_t b) { return (b + 255) / 256 * 256; }

const KernelSet *kernels_for(int pde, int dim, int N, int prec)
{
    if (N < 1 || N > 9) return nullptr;
    return lookup_kernels(pde, dim, N, prec);
}

int nvar_of(int pde, int dim) { return pde_nvar(pde, dim); }

// ---------------------------------------------------------------------------
// device memory: the caller's allocator hook, else stream-ordered cudaMallocAsync
// ---------------------------------------------------------------------------
struct Mem {
    aderdg_alloc_t hook{};
    bool has_hook = false;
    cudaStream_t st = nullptr;
    size_t in_use = 0;
    void *get(size_t bytes)
    {
        bytes = a256(bytes);
        void *p = nullptr;
        if (has_hook) p = hook.alloc(bytes, hook.ctx);
        else if (cudaMallocAsync(&p, bytes, st) != cudaSuccess) { cudaGetLastError(); p = nullptr; }
        if (p) in_use += bytes;
        return p;
    }
    void put(void *p, size_t bytes)
    {
        if (!p) return;
        if (has_hook) hook.free(p, hook.ctx);
        else cudaFreeAsync(p, st);
        in_use -= a256(bytes);
    }
};

struct Slot {
    int pde = 0, dim = 0, N = 0, M = 0, NS = 0, NF = 0, NREC = 0, picard = 0, guess = 0, prec = 0;
    long long E = 0;
    int cells[3] = {1, 1, 1};
    double inv_dx[3] = {1, 1, 1}, vol = 1;
    PdeParams pp{};
    double alpha = 0;
    const KernelSet *ks = nullptr;
    void *block = nullptr;  // u | V | traces
    size_t bytes = 0;
    double *u = nullptr;
    void *V = nullptr, *tr = nullptr;
    double *ref = nullptr;
    void *qprev = nullptr;     // extrapolation guess: last predictor
    // subcell limiter (FP64): u^n, extremes of u^n and of the candidate, flags
    bool limiter = false;
    LimKernels lk{};
    double *u_prev = nullptr, *lim_mm = nullptr, *lim_mmc = nullptr;
    int *lim_flags = nullptr, *lim_list = nullptr;
    double *lim_fb = nullptr;  // troubled elements' face fluxes for the coupling
    int *lim_slot = nullptr;
    long long lim_fb_slots = 0;
    int ctl_index = -1;
    // placement in the current group arrays (for k_cfl)
    int group = -1, member = -1;
};

size_t lim_bytes(const Slot &s)
{
    const size_t ns = (size_t)s.E * s.NS * s.M;
    const size_t fb = s.lim_fb_slots > 0 ? a256((size_t)s.lim_fb_slots * limiter_flux_doubles(s.dim, s.N, s.M, s.ks->ncp != 0) * 8) +
                                               a256((size_t)s.E * 4)
                                         : 0;
    return s.limiter ? a256(ns * 8) + 2 * a256((size_t)s.E * s.M * 2 * 8) + 2 * a256((size_t)s.E * 4) + fb : 0;
}

size_t slot_bytes(const Slot &s)
{
    const size_t ns = (size_t)s.E * s.NS * s.M;
    return a256(ns * 8) + a256(ns * s.ks->elem_bytes) + a256((size_t)s.E * s.NREC * s.ks->rs * s.ks->elem_bytes) +
           a256((size_t)s.E * s.ks->rf * 8) + (s.guess == ADERDG_GUESS_EXTRAP ? a256(ns * (s.N + 1) * s.ks->elem_bytes) : 0) +
           lim_bytes(s);
}

int make_slot(const aderdg_solve_spec_t &sp, int prec, int guess, int picard, double alpha, Slot &s,
              bool limiter = false)
{
    const aderdg_mesh_t &m = sp.mesh;
    long long E = 0;
    const char *why = nullptr;
    if (check_mesh(m, sp.pde.kind, &E, &why)) return fail(ADERDG_E_INVAL, why);
    const int M = nvar_of(sp.pde.kind, m.dim);
    const KernelSet *ks = kernels_for(sp.pde.kind, m.dim, sp.N, prec);
    if (!ks) return fail(ADERDG_E_UNSUPPORTED, "no kernels compiled for this (pde, dim, N)");
    if (check_pde_params(sp.pde, &why)) return fail(ADERDG_E_INVAL, why);
    if (guess < ADERDG_GUESS_TRIVIAL || guess > ADERDG_GUESS_CERK) return fail(ADERDG_E_INVAL, "bad initial guess");
    LimKernels lk{};
    if (limiter) {
        const int rc = limiter_kernels(sp.pde.kind, m.dim, sp.N, prec, guess, false, &lk, &why);
        if (rc) return fail(rc, why);
    }
    s = Slot();
    s.limiter = limiter;
    s.lk = lk;
    s.pde = sp.pde.kind;
    s.dim = m.dim;
    s.N = sp.N;
    s.M = M;
    s.NS = ipow(sp.N + 1, m.dim);
    s.NF = ipow(sp.N + 1, m.dim - 1);
    s.NREC = m.dim * 2 * s.NF;
    s.guess = guess;
    s.prec = prec;
    s.picard = picard > 0 ? picard : default_picard(sp.N, guess);
    s.alpha = alpha > 0 ? alpha : default_alpha(sp.N);
    s.ks = ks;
    s.E = E;
    for (int d = 0; d < m.dim; ++d) {
        s.cells[d] = (int)m.cells[d];
        const double dx = (m.hi[d] - m.lo[d]) / m.cells[d];
        s.inv_dx[d] = 1.0 / dx;
        s.vol *= dx;
    }
    for (int i = 0; i < 8; ++i) s.pp.p[i] = sp.pde.p[i];
    fill_pde_consts(s.pde, s.pp);
    s.lim_fb_slots = limiter ? limiter_flux_slots(E, s.dim, s.N, s.M, ks->ncp != 0) : 0;
    s.bytes = slot_bytes(s);
    return ADERDG_OK;
}

__global__ void k_dt_batch(Control *const *ctls, int count)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) dt_update(ctls[i]);
}


__global__ void k_set_tend(Control *const *ctls, const double *t_end, int count)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) ctls[i]->t_end = t_end[i];
}

struct Group {
    int pde = 0, dim = 0, N = 0, prec = 0;
    bool extrap = false;  // its solves use the extrapolation or CERK guess (predictor variant)
    bool limiter = false;  // its solves run the subcell limiter
    long long elems = 0;   // elements of all its solves
    PdeParams pp{};
    const KernelSet *ks = nullptr;  // compiled kernels of the group
    KernelSet kso{};                // the same with the tile shapes in use
    KParams kp{};
    std::vector<Slot *> members;
    SolveDesc *d_desc = nullptr;
    int cap = 0;
    long long ntp = 0, ntc = 0;
};

// solves share a group (one predictor and one corrector launch) when they
// have the same kernels (PDE, dimension, order, precision) and parameters
bool same_group(const Group &g, const Slot &s)
{
    return g.ks == s.ks && g.pde == s.pde && g.dim == s.dim && g.N == s.N && g.prec == s.prec &&
           g.extrap == (s.guess == ADERDG_GUESS_EXTRAP || s.guess == ADERDG_GUESS_CERK) && g.limiter == s.limiter &&
           std::memcmp(&g.pp, &s.pp, sizeof(PdeParams)) == 0;
}

class Engine {
public:
    Mem mem;
    cudaStream_t st = nullptr;
    int pred_req = 0, corr_req = 0;  // requested tile shapes (index or ADERDG_SHAPE_AUTOTUNE)
    std::string tune_cache;          // empty: none
    int device = 0;
    // control blocks: one pool, slots index into it
    Control *d_ctl = nullptr;
    Control *h_ctl = nullptr;  // pinned mirror
    int ctl_cap = 0;
    std::vector<int> ctl_free;
    std::vector<Slot *> active;
    std::vector<Group> groups;
    Control **d_ctlptrs = nullptr;
    double *d_tend = nullptr;
    int ptr_cap = 0;
    bool dirty = true;
    cudaGraphExec_t graph = nullptr;
    int graph_steps = 0;
    // limited groups: the copies of u^n and their subcell extremes run on a
    // second stream beside the group's predictor (event fork and join)
    cudaStream_t side = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;

    int init(int capacity, cudaStream_t stream, const aderdg_alloc_t *hook)
    {
        cudaGetDevice(&device);
        st = stream;
        mem.st = stream;
        CKB(cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking));
        CKB(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
        CKB(cudaEventCreateWithFlags(&join, cudaEventDisableTiming));
        if (hook) { mem.hook = *hook; mem.has_hook = true; }
        ctl_cap = std::max(1, capacity);
        d_ctl = (Control *)mem.get(sizeof(Control) * ctl_cap);
        if (!d_ctl) return fail(ADERDG_E_NOMEM, "control pool allocation failed");
        CKB(cudaMallocHost(&h_ctl, sizeof(Control) * ctl_cap));
        for (int i = ctl_cap - 1; i >= 0; --i) ctl_free.push_back(i);
        return ADERDG_OK;
    }

    void release()
    {
        if (st) cudaStreamSynchronize(st);
        if (graph) cudaGraphExecDestroy(graph);
        graph = nullptr;
        for (Slot *s : active) { mem.put(s->block, s->bytes); delete s; }
        active.clear();
        for (Group &g : groups) mem.put(g.d_desc, sizeof(SolveDesc) * g.cap);
        groups.clear();
        mem.put(d_ctlptrs, sizeof(Control *) * ptr_cap);
        mem.put(d_tend, sizeof(double) * ptr_cap);
        mem.put(d_ctl, sizeof(Control) * ctl_cap);
        if (h_ctl) cudaFreeHost(h_ctl);
        if (st) cudaStreamSynchronize(st);
        if (side) cudaStreamSynchronize(side);
        if (fork) cudaEventDestroy(fork);
        if (join) cudaEventDestroy(join);
        if (side) cudaStreamDestroy(side);
        fork = join = nullptr;
        side = nullptr;
        h_ctl = nullptr;
        d_ctl = nullptr;
    }

    Control *ctl_of(const Slot *s) const { return d_ctl + s->ctl_index; }

    // allocate a slot's buffers and control block; state zero, t = t0
    int add(Slot *s, double t0)
    {
        if (ctl_free.empty()) return fail(ADERDG_E_BUSY, "no free control block");
        s->block = mem.get(s->bytes);
        if (!s->block) return fail(ADERDG_E_NOMEM, "slot allocation failed");
        const size_t ns = (size_t)s->E * s->NS * s->M;
        unsigned char *b = static_cast<unsigned char *>(s->block);
        s->u = reinterpret_cast<double *>(b);
        s->V = b + a256(ns * 8);
        s->tr = b + a256(ns * 8) + a256(ns * s->ks->elem_bytes);
        const size_t o_ref = a256(ns * 8) + a256(ns * s->ks->elem_bytes) +
                             a256((size_t)s->E * s->NREC * s->ks->rs * s->ks->elem_bytes);
        s->ref = s->ks->rf > 0 ? reinterpret_cast<double *>(b + o_ref) : nullptr;
        s->qprev = s->guess == ADERDG_GUESS_EXTRAP ? b + o_ref + a256((size_t)s->E * s->ks->rf * 8) : nullptr;
        if (s->limiter) {
            unsigned char *l = b + s->bytes - lim_bytes(*s);
            s->u_prev = reinterpret_cast<double *>(l);
            s->lim_mm = reinterpret_cast<double *>(l + a256(ns * 8));
            s->lim_mmc = reinterpret_cast<double *>(l + a256(ns * 8) + a256((size_t)s->E * s->M * 2 * 8));
            s->lim_flags = reinterpret_cast<int *>(l + a256(ns * 8) + 2 * a256((size_t)s->E * s->M * 2 * 8));
            s->lim_list = reinterpret_cast<int *>(reinterpret_cast<unsigned char *>(s->lim_flags) +
                                                  a256((size_t)s->E * 4));
            if (s->lim_fb_slots > 0) {
                unsigned char *f = reinterpret_cast<unsigned char *>(s->lim_list) + a256((size_t)s->E * 4);
                s->lim_fb = reinterpret_cast<double *>(f);
                s->lim_slot = reinterpret_cast<int *>(
                    f + a256((size_t)s->lim_fb_slots * limiter_flux_doubles(s->dim, s->N, s->M, s->ks->ncp != 0) * 8));
            }
            CKB(cudaMemsetAsync(s->lim_flags, 0, sizeof(int) * (size_t)s->E, st));
        }
        s->ctl_index = ctl_free.back();
        ctl_free.pop_back();
        Control c;
        std::memset(&c, 0, sizeof(c));
        c.t = t0;
        c.t_end = t0;
        c.alpha = s->alpha;
        c.dim = s->dim;
        for (int d = 0; d < 3; ++d) c.inv_dx[d] = s->inv_dx[d];
        std::memcpy(&h_ctl[s->ctl_index], &c, sizeof(c));
        CKB(cudaMemcpyAsync(ctl_of(s), &h_ctl[s->ctl_index], sizeof(c), cudaMemcpyHostToDevice, st));
        active.push_back(s);
        dirty = true;
        return ADERDG_OK;
    }

    void remove(Slot *s)
    {
        auto it = std::find(active.begin(), active.end(), s);
        if (it != active.end()) active.erase(it);
        mem.put(s->block, s->bytes);
        ctl_free.push_back(s->ctl_index);
        delete s;
        dirty = true;
    }

    // group arrays, tile offsets and the control-pointer array
    int rebuild()
    {
        if (!dirty) return ADERDG_OK;
        if (graph) { cudaGraphExecDestroy(graph); graph = nullptr; }
        std::vector<Group> ng;
        for (Slot *s : active) {
            int gi = -1;
            for (size_t i = 0; i < ng.size(); ++i)
                if (same_group(ng[i], *s)) { gi = (int)i; break; }
            if (gi < 0) {
                Group g;
                g.pde = s->pde; g.dim = s->dim; g.N = s->N; g.prec = s->prec; g.pp = s->pp; g.ks = s->ks;
                g.extrap = s->guess == ADERDG_GUESS_EXTRAP || s->guess == ADERDG_GUESS_CERK;
                g.limiter = s->limiter;
                ng.push_back(g);
                gi = (int)ng.size() - 1;
            }
            s->group = gi;
            s->member = (int)ng[gi].members.size();
            ng[gi].members.push_back(s);
            ng[gi].elems += s->E;
        }
        // tile shapes per group (may autotune on first use of a key)
        for (Group &g : ng) {
            const int rc = resolve_shapes(g.ks, g.pde, g.dim, g.N, g.prec, g.pp, pred_req, corr_req,
                                          tune_cache.empty() ? nullptr : tune_cache.c_str(), g.extrap, &g.kso);
            if (rc) return rc;
        }
        // reuse device descriptor arrays of old groups where possible
        for (Group &g : groups) mem.put(g.d_desc, sizeof(SolveDesc) * g.cap);
        groups.clear();
        for (Group &g : ng) {
            std::vector<SolveDesc> h(g.members.size());
            long long tp = 0, tc = 0;
            for (size_t i = 0; i < g.members.size(); ++i) {
                const Slot *s = g.members[i];
                SolveDesc &d = h[i];
                std::memset(&d, 0, sizeof(d));
                d.E = s->E;
                d.tile0_p = tp;
                d.tile0_c = tc;
                tp += (s->E + g.kso.pred_epb - 1) / g.kso.pred_epb;
                tc += (s->E + g.kso.corr_epb - 1) / g.kso.corr_epb;
                for (int k = 0; k < 3; ++k) { d.cells[k] = s->cells[k]; d.inv_dx[k] = s->inv_dx[k]; }
                fill_desc_spacing(d);
                fill_desc_lift(d, s->N);
                d.picard = s->picard;
                d.guess = s->guess;
                d.picard_first = default_picard(s->N, ADERDG_GUESS_ORDER3);
                d.qprev = s->qprev;
                d.u = s->u;
                d.u_out = s->u;
                d.V = s->V;
                d.tr = s->tr;
                d.ref = s->ref;
                d.ctl = ctl_of(s);
                d.u_prev = s->u_prev;
                d.lim_mm = s->lim_mm;
                d.lim_mmc = s->lim_mmc;
                d.lim_flags = s->lim_flags;
                d.lim_list = s->lim_list;
                d.lim_fb = s->lim_fb;
                d.lim_slot = s->lim_slot;
                d.lim_fb_slots = s->lim_fb_slots;
            }
            g.ntp = tp;
            g.ntc = tc;
            g.cap = (int)h.size();
            g.d_desc = (SolveDesc *)mem.get(sizeof(SolveDesc) * g.cap);
            if (!g.d_desc) return fail(ADERDG_E_NOMEM, "descriptor allocation failed");
            CKB(cudaMemcpyAsync(g.d_desc, h.data(), sizeof(SolveDesc) * h.size(), cudaMemcpyHostToDevice, st));
            std::memset(&g.kp, 0, sizeof(g.kp));
            g.kp.solves = g.d_desc;
            g.kp.nsolves = (int)h.size();
            g.kp.use_ctl_dt = 1;
            g.kp.pde = g.pp;
            if (build_basis(g.N, g.kp.b)) return fail(ADERDG_E_INVAL, "basis construction failed");
            fill_ops(g.kp);
            groups.push_back(g);
        }
        // control pointers in active order
        if ((int)active.size() > ptr_cap) {
            mem.put(d_ctlptrs, sizeof(Control *) * ptr_cap);
            mem.put(d_tend, sizeof(double) * ptr_cap);
            ptr_cap = std::max<int>((int)active.size(), 2 * ptr_cap);
            d_ctlptrs = (Control **)mem.get(sizeof(Control *) * ptr_cap);
            d_tend = (double *)mem.get(sizeof(double) * ptr_cap);
            if (!d_ctlptrs || !d_tend) return fail(ADERDG_E_NOMEM, "pointer array allocation failed");
        }
        std::vector<Control *> hp(active.size());
        for (size_t i = 0; i < active.size(); ++i) hp[i] = ctl_of(active[i]);
        if (!hp.empty())
            CKB(cudaMemcpyAsync(d_ctlptrs, hp.data(), sizeof(Control *) * hp.size(), cudaMemcpyHostToDevice, st));
        CKB(cudaStreamSynchronize(st));  // host staging vectors go out of scope
        dirty = false;
        return ADERDG_OK;
    }

    int set_state(Slot *s, const double *u, int where, double t)
    {
        int rc = rebuild();
        if (rc) return rc;
        const size_t bytes = (size_t)s->E * s->NS * s->M * sizeof(double);
        CKB(cudaMemcpyAsync(s->u, u, bytes, where == ADERDG_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                            st));
        Control &c = h_ctl[s->ctl_index];
        std::memset(&c, 0, sizeof(c));
        c.t = t;
        c.t_end = t;  // no step until a t_end is given
        c.alpha = s->alpha;
        c.dim = s->dim;
        for (int d = 0; d < 3; ++d) c.inv_dx[d] = s->inv_dx[d];
        CKB(cudaMemcpyAsync(ctl_of(s), &c, sizeof(c), cudaMemcpyHostToDevice, st));
        const Group &g = groups[s->group];
        KParams kp = g.kp;
        kp.solves = g.d_desc + s->member;
        kp.nsolves = 1;
        const long long blocks = std::min<long long>(4 * 152, (s->E * s->NS + 255) / 256);
        s->ks->cfl<<<(unsigned)blocks, 256, 0, st>>>(kp);
        CKB(cudaGetLastError());
        return ADERDG_OK;
    }

    int set_tend(const double *t_end)
    {
        int rc = rebuild();
        if (rc) return rc;
        if (active.empty()) return ADERDG_OK;
        CKB(cudaMemcpyAsync(d_tend, t_end, sizeof(double) * active.size(), cudaMemcpyHostToDevice, st));
        k_set_tend<<<(unsigned)((active.size() + 127) / 128), 128, 0, st>>>(d_ctlptrs, d_tend, (int)active.size());
        CKB(cudaGetLastError());
        CKB(cudaStreamSynchronize(st));  // the host array may be temporary
        return ADERDG_OK;
    }

    int enqueue_step()
    {
        if (active.empty()) return ADERDG_OK;
        k_dt_batch<<<(unsigned)((active.size() + 127) / 128), 128, 0, st>>>(d_ctlptrs, (int)active.size());
        CKB(cudaGetLastError());
        for (Group &g : groups) {
            KParams kp = g.kp;
            const LimKernels *glk = g.limiter ? &g.members[0]->lk : nullptr;  // one (PDE, d, N, precision) per group
            if (g.limiter) {
                // u^n for the limiter (before the corrector overwrites it) and
                // its subcell extremes, on the side stream beside the predictor
                CKB(cudaEventRecord(fork, st));
                CKB(cudaStreamWaitEvent(side, fork, 0));
                for (const Slot *m : g.members)
                    CKB(cudaMemcpyAsync(m->u_prev, m->u, (size_t)m->E * m->NS * m->M * sizeof(double),
                                        cudaMemcpyDeviceToDevice, side));
                glk->minmax<<<glk->minmax_grid(g.elems), 128, glk->smem_w, side>>>(kp);
                CKB(cudaEventRecord(join, side));
            }
            kp.ntiles = g.ntp;
            g.kso.predictor<<<(unsigned)g.ntp, g.kso.pred_threads, g.kso.pred_smem, st>>>(kp);
            if (g.limiter) CKB(cudaStreamWaitEvent(st, join, 0));
            kp.ntiles = g.ntc;
            g.kso.corrector<<<(unsigned)g.ntc, g.kso.corr_threads, g.kso.corr_smem, st>>>(kp);
            if (g.limiter) {
                // one launch of each limiter kernel for all solves of the group
                const KernelSet *ks = g.ks;
                const LimKernels &lk = *glk;
                const unsigned grid = (unsigned)std::min<long long>(g.elems, 152LL * 16);
                lk.detect<<<grid, 128, lk.smem_w, st>>>(kp);
                lk.fv<<<grid, 128, lk.smem, st>>>(kp);
                lk.couple<<<grid, 128, lk.smem, st>>>(kp);
                for (const Slot *m : g.members) {
                    KParams k1 = g.kp;
                    k1.solves = g.d_desc + m->member;
                    k1.nsolves = 1;
                    k1.use_ctl_dt = 1;
                    k1.lim_pass = 1;  // the wave speeds of a limited state that changed
                    ks->cfl<<<(unsigned)std::min<long long>(4 * 152, (m->E * m->NS + 255) / 256), 256, 0, st>>>(k1);
                }
            }
        }
        CKB(cudaGetLastError());
        return ADERDG_OK;
    }

    // k steps, as a replayed graph when k matches the captured length
    int steps(int k)
    {
        int rc = rebuild();
        if (rc) return rc;
        constexpr int CHUNK = 8;
        if (k == CHUNK && !graph && st) {
            cudaStreamCaptureStatus cs;
            if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone &&
                cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
                bool ok = true;
                for (int i = 0; i < CHUNK && ok; ++i) ok = enqueue_step() == ADERDG_OK;
                cudaGraph_t gr = nullptr;
                if (cudaStreamEndCapture(st, &gr) != cudaSuccess) ok = false;
                if (ok && cudaGraphInstantiate(&graph, gr, 0) != cudaSuccess) graph = nullptr;
                if (gr) cudaGraphDestroy(gr);
            }
            cudaGetLastError();
        }
        if (graph && k == CHUNK) {
            CKB(cudaGraphLaunch(graph, st));
            return ADERDG_OK;
        }
        for (int i = 0; i < k; ++i) {
            rc = enqueue_step();
            if (rc) return rc;
        }
        return ADERDG_OK;
    }

    // copy the control pool to the pinned mirror and wait
    int read_controls()
    {
        int hi = 0;
        for (Slot *s : active) hi = std::max(hi, s->ctl_index + 1);
        if (hi > 0) CKB(cudaMemcpyAsync(h_ctl, d_ctl, sizeof(Control) * hi, cudaMemcpyDeviceToHost, st));
        CKB(cudaStreamSynchronize(st));
        return ADERDG_OK;
    }
};

}  // namespace

// ===========================================================================
// batch API
// ===========================================================================

struct aderdg_batch_s {
    Engine eng;
    std::vector<Slot *> slots;  // by index
    std::vector<double> t_end;
    bool own_stream = false;
    int64_t dofs = 0;
};

extern "C" {

int aderdg_batch_create(const aderdg_solve_spec_t *specs, int count, const aderdg_config_t *cfg,
                        aderdg_batch_t **out)
{
    if (!out) return fail(ADERDG_E_INVAL, "out is NULL");
    *out = nullptr;
    if (!specs || count <= 0) return fail(ADERDG_E_INVAL, "need count > 0 specs");
    const int prec = cfg ? cfg->precision : ADERDG_FP64;
    if (prec != ADERDG_FP64 && prec != ADERDG_MIXED_FP32) return fail(ADERDG_E_INVAL, "bad precision");
    if (cfg && !valid_shape_requests(cfg->pred_shape, cfg->corr_shape))
        return fail(ADERDG_E_INVAL, "bad tile shape request");
    if (cfg && (cfg->limiter < 0 || cfg->limiter > 2)) return fail(ADERDG_E_INVAL, "limiter must be 0, 1 or 2");
    if (cfg && cfg->limiter == 2)
        return fail(ADERDG_E_UNSUPPORTED, "kept subcell data (limiter 2) is available on single-solve handles");
    std::vector<Slot> tmp(count);
    for (int i = 0; i < count; ++i) {
        int rc = make_slot(specs[i], prec, cfg ? cfg->initial_guess : 0, cfg ? cfg->picard_iters : 0,
                           cfg ? cfg->cfl_alpha : 0.0, tmp[i], cfg && cfg->limiter);
        if (rc) return rc;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return fail(ADERDG_E_CUDA, "no CUDA device available (the library has no CPU path)");
    }
    aderdg_batch_t *b = new aderdg_batch_s();
    cudaStream_t st = cfg && cfg->cuda_stream ? (cudaStream_t)cfg->cuda_stream : nullptr;
    if (!st) {
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            delete b;
            return fail(ADERDG_E_CUDA, "cudaStreamCreate failed");
        }
        b->own_stream = true;
    }
    int rc = b->eng.init(count, st, cfg ? cfg->alloc : nullptr);
    if (cfg) {
        b->eng.pred_req = cfg->pred_shape;
        b->eng.corr_req = cfg->corr_shape;
        if (cfg->tune_cache) b->eng.tune_cache = cfg->tune_cache;
    }
    for (int i = 0; rc == ADERDG_OK && i < count; ++i) {
        Slot *s = new Slot(tmp[i]);
        rc = b->eng.add(s, 0.0);
        if (rc) { delete s; break; }
        b->slots.push_back(s);
        b->dofs += s->E * s->NS;
        // zero state
        if (cudaMemsetAsync(s->u, 0, (size_t)s->E * s->NS * s->M * 8, st) != cudaSuccess) rc = ADERDG_E_CUDA;
    }
    if (rc == ADERDG_OK) rc = b->eng.rebuild();
    if (rc) {
        std::string m = aderdg_last_error();
        aderdg_batch_destroy(b);
        return fail(rc, m);
    }
    b->t_end.assign(count, 0.0);
    *out = b;
    return ADERDG_OK;
}

int aderdg_batch_destroy(aderdg_batch_t *b)
{
    if (!b) return ADERDG_OK;
    cudaStream_t st = b->eng.st;
    b->eng.release();
    if (b->own_stream && st) cudaStreamDestroy(st);
    delete b;
    return ADERDG_OK;
}

int aderdg_batch_set_state(aderdg_batch_t *b, int i, const double *u, int where, double t)
{
    if (!b || !u || i < 0 || i >= (int)b->slots.size()) return fail(ADERDG_E_INVAL, "bad batch index");
    if (!std::isfinite(t)) return fail(ADERDG_E_INVAL, "t must be finite");
    int rc = b->eng.set_state(b->slots[i], u, where, t);
    if (rc) return rc;
    CKB(cudaStreamSynchronize(b->eng.st));
    return ADERDG_OK;
}

int aderdg_batch_get_state(aderdg_batch_t *b, int i, double *u, int where, double *t, int64_t *step)
{
    if (!b || !u || i < 0 || i >= (int)b->slots.size()) return fail(ADERDG_E_INVAL, "bad batch index");
    Slot *s = b->slots[i];
    const size_t bytes = (size_t)s->E * s->NS * s->M * sizeof(double);
    CKB(cudaMemcpyAsync(u, s->u, bytes, where == ADERDG_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                        b->eng.st));
    int rc = b->eng.read_controls();
    if (rc) return rc;
    const Control &c = b->eng.h_ctl[s->ctl_index];
    if (t) *t = c.t;
    if (step) *step = c.step;
    if (c.flags & FLAG_NONFINITE) return fail(ADERDG_E_NONFINITE, "non-finite value in the state");
    return ADERDG_OK;
}

int aderdg_batch_step(aderdg_batch_t *b, const double *t_end)
{
    if (!b) return fail(ADERDG_E_INVAL, "NULL batch");
    // the engine orders controls by its active list = slot order here; the
    // host copy of t_end is re-sent every call (set_state resets the device's)
    if (t_end)
        for (size_t i = 0; i < b->slots.size(); ++i) b->t_end[i] = t_end[i];
    int rc = b->eng.set_tend(b->t_end.data());
    if (rc) return rc;
    return b->eng.steps(1);
}

int aderdg_batch_advance(aderdg_batch_t *b, const double *t_end, int64_t max_steps)
{
    if (!b || max_steps < 0) return fail(ADERDG_E_INVAL, "bad arguments");
    if (t_end)
        for (size_t i = 0; i < b->slots.size(); ++i) b->t_end[i] = t_end[i];
    {
        int rc = b->eng.set_tend(b->t_end.data());
        if (rc) return rc;
    }
    int64_t done = 0;
    bool bad = false;
    while (done < max_steps) {
        const int k = (int)std::min<int64_t>(8, max_steps - done);
        int rc = b->eng.steps(k);
        if (rc) return rc;
        done += k;
        rc = b->eng.read_controls();
        if (rc) return rc;
        bool all = true;
        for (Slot *s : b->slots) {
            const Control &c = b->eng.h_ctl[s->ctl_index];
            if (c.flags & FLAG_NONFINITE) { bad = true; continue; }
            if (c.t < c.t_end) all = false;
        }
        if (all) break;
    }
    if (bad) return fail(ADERDG_E_NONFINITE, "a solve produced a non-finite value");
    return ADERDG_OK;
}

int aderdg_batch_info(const aderdg_batch_t *b, int64_t *dofs, size_t *device_bytes, int *groups)
{
    if (!b) return fail(ADERDG_E_INVAL, "NULL batch");
    if (dofs) *dofs = b->dofs;
    if (device_bytes) *device_bytes = b->eng.mem.in_use;
    if (groups) *groups = (int)b->eng.groups.size();
    return ADERDG_OK;
}

int aderdg_batch_troubled(aderdg_batch_t *b, int i, int *flags, int64_t *count)
{
    if (!b || i < 0 || i >= (int)b->slots.size()) return fail(ADERDG_E_INVAL, "bad batch index");
    const Slot *s = b->slots[i];
    if (!s->limiter) return fail(ADERDG_E_INVAL, "the batch has no limiter");
    std::vector<int> f((size_t)s->E);
    CKB(cudaMemcpyAsync(f.data(), s->lim_flags, sizeof(int) * (size_t)s->E, cudaMemcpyDeviceToHost, b->eng.st));
    CKB(cudaStreamSynchronize(b->eng.st));
    int64_t c = 0;
    for (long long e = 0; e < s->E; ++e) c += f[(size_t)e] != 0;
    if (flags) std::memcpy(flags, f.data(), sizeof(int) * (size_t)s->E);
    if (count) *count = c;
    return ADERDG_OK;
}

int aderdg_batch_status(aderdg_batch_t *b, int *status)
{
    if (!b || !status) return fail(ADERDG_E_INVAL, "NULL argument");
    int rc = b->eng.read_controls();
    if (rc) return rc;
    for (size_t i = 0; i < b->slots.size(); ++i) {
        const Control &c = b->eng.h_ctl[b->slots[i]->ctl_index];
        status[i] = (c.flags & FLAG_NONFINITE) ? ADERDG_E_NONFINITE : (c.t < c.t_end ? 0 : 1);
    }
    return ADERDG_OK;
}

}  // extern "C"

// ===========================================================================
// server
// ===========================================================================

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t ticket = 0;
    Slot spec;                 // sizes, kernels (buffers not allocated yet)
    std::vector<double> u0;
    double t_end = 0;
    Clock::time_point submitted, admitted, finished;
    int status = ADERDG_PENDING;
    bool cancelled = false;
    Slot *slot = nullptr;      // while admitted
    std::vector<double> result;
    double t = 0;
    int64_t steps = 0;
};

}  // namespace

struct aderdg_server_s {
    Engine eng;
    bool own_stream = false;
    size_t budget = 0;
    int max_queue = 100000;
    int steps_per_round = 8;
    int prec = ADERDG_FP64;
    int guess = ADERDG_GUESS_TRIVIAL;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Request *> queue;                         // submitted, not admitted
    std::vector<Request *> running;                      // admitted
    std::unordered_map<uint64_t, Request *> tickets;     // all live tickets
    uint64_t next_ticket = 1;
    int64_t finished = 0;
    bool stop = false;
    std::thread worker;
    int worker_error = 0;
    size_t slot_bytes_in_use = 0;  // what the budget counts (state, volume, traces)

    void loop();
};

void aderdg_server_s::loop()
{
    cudaSetDevice(eng.device);
    std::vector<Request *> newly;
    while (true) {
        newly.clear();
        {
            std::unique_lock<std::mutex> lk(mu);
            if (running.empty() && queue.empty())
                cv.wait_for(lk, std::chrono::milliseconds(20), [&] { return stop || !queue.empty(); });
            if (stop) break;
            // drop cancelled queued requests
            for (auto it = queue.begin(); it != queue.end();) {
                if ((*it)->cancelled) { (*it)->status = ADERDG_E_CANCELLED; (*it)->finished = Clock::now(); it = queue.erase(it); }
                else ++it;
            }
            // admission: oldest first while the budget allows
            while (!queue.empty()) {
                Request *r = queue.front();
                if (slot_bytes_in_use + r->spec.bytes > budget || eng.ctl_free.empty()) break;
                slot_bytes_in_use += r->spec.bytes;
                queue.pop_front();
                newly.push_back(r);
            }
        }
        for (Request *r : newly) {
            Slot *s = new Slot(r->spec);
            if (eng.add(s, 0.0) != ADERDG_OK) {
                delete s;
                std::lock_guard<std::mutex> lk(mu);
                slot_bytes_in_use -= r->spec.bytes;
                r->status = ADERDG_E_NOMEM;
                r->finished = Clock::now();
                continue;
            }
            r->slot = s;
            if (eng.set_state(s, r->u0.data(), ADERDG_HOST, 0.0) != ADERDG_OK) { worker_error = ADERDG_E_CUDA; break; }
            std::vector<double>().swap(r->u0);
            std::lock_guard<std::mutex> lk(mu);
            r->admitted = Clock::now();
            running.push_back(r);
        }
        if (worker_error) break;
        if (running.empty()) continue;
        // t_end per active slot, in the engine's active order
        {
            std::vector<double> te(eng.active.size());
            std::unordered_map<Slot *, double> m;
            {
                std::lock_guard<std::mutex> lk(mu);
                for (Request *r : running) m[r->slot] = r->cancelled ? 0.0 : r->t_end;
            }
            for (size_t i = 0; i < eng.active.size(); ++i) te[i] = m[eng.active[i]];
            if (eng.set_tend(te.data()) != ADERDG_OK) { worker_error = ADERDG_E_CUDA; break; }
        }
        if (eng.steps(steps_per_round) != ADERDG_OK || eng.read_controls() != ADERDG_OK) {
            worker_error = ADERDG_E_CUDA;
            break;
        }
        // retire finished / failed / cancelled solves
        std::vector<Request *> done;
        {
            std::lock_guard<std::mutex> lk(mu);
            for (Request *r : running) {
                const Control &c = eng.h_ctl[r->slot->ctl_index];
                if (r->cancelled || (c.flags & FLAG_NONFINITE) || !(c.t < c.t_end)) done.push_back(r);
            }
        }
        for (Request *r : done) {
            const Control c = eng.h_ctl[r->slot->ctl_index];
            const size_t nv = (size_t)r->slot->E * r->slot->NS * r->slot->M;
            int status = ADERDG_OK;
            if (r->cancelled) status = ADERDG_E_CANCELLED;
            else if (c.flags & FLAG_NONFINITE) status = ADERDG_E_NONFINITE;
            else {
                r->result.resize(nv);
                if (cudaMemcpyAsync(r->result.data(), r->slot->u, nv * 8, cudaMemcpyDeviceToHost, eng.st) != cudaSuccess ||
                    cudaStreamSynchronize(eng.st) != cudaSuccess)
                    status = ADERDG_E_CUDA;
            }
            eng.remove(r->slot);
            std::lock_guard<std::mutex> lk(mu);
            slot_bytes_in_use -= r->spec.bytes;
            r->slot = nullptr;
            r->t = c.t;
            r->steps = c.step;
            r->finished = Clock::now();
            r->status = status;
            running.erase(std::find(running.begin(), running.end(), r));
            ++finished;
        }
    }
    // drain: stop requested or a CUDA error
    std::lock_guard<std::mutex> lk(mu);
    for (Request *r : running) {
        if (r->slot) { eng.remove(r->slot); r->slot = nullptr; }
        if (r->status == ADERDG_PENDING) r->status = worker_error ? worker_error : ADERDG_E_CANCELLED;
    }
    running.clear();
    for (Request *r : queue)
        if (r->status == ADERDG_PENDING) r->status = worker_error ? worker_error : ADERDG_E_CANCELLED;
    queue.clear();
}

extern "C" {

int aderdg_server_create(const aderdg_server_config_t *cfg, aderdg_server_t **out)
{
    if (!out) return fail(ADERDG_E_INVAL, "out is NULL");
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return fail(ADERDG_E_CUDA, "no CUDA device available (the library has no CPU path)");
    }
    aderdg_server_t *s = new aderdg_server_s();
    s->prec = cfg ? cfg->precision : ADERDG_FP64;
    if (s->prec != ADERDG_FP64 && s->prec != ADERDG_MIXED_FP32) { delete s; return fail(ADERDG_E_INVAL, "bad precision"); }
    if (cfg && !valid_shape_requests(cfg->pred_shape, cfg->corr_shape)) {
        delete s;
        return fail(ADERDG_E_INVAL, "bad tile shape request");
    }
    s->guess = cfg ? cfg->initial_guess : ADERDG_GUESS_TRIVIAL;
    if (s->guess < ADERDG_GUESS_TRIVIAL || s->guess > ADERDG_GUESS_CERK) {
        delete s;
        return fail(ADERDG_E_INVAL, "bad initial guess");
    }
    if (cfg && cfg->max_queue > 0) s->max_queue = cfg->max_queue;
    if (cfg && cfg->steps_per_round > 0) s->steps_per_round = cfg->steps_per_round;
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    s->budget = (cfg && cfg->device_budget_bytes) ? cfg->device_budget_bytes : (size_t)(0.9 * free_b);
    cudaStream_t st = cfg && cfg->cuda_stream ? (cudaStream_t)cfg->cuda_stream : nullptr;
    if (!st) {
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            delete s;
            return fail(ADERDG_E_CUDA, "cudaStreamCreate failed");
        }
        s->own_stream = true;
    }
    int rc = s->eng.init(4096, st, nullptr);
    if (cfg) {
        s->eng.pred_req = cfg->pred_shape;
        s->eng.corr_req = cfg->corr_shape;
        if (cfg->tune_cache) s->eng.tune_cache = cfg->tune_cache;
    }
    if (rc) {
        std::string m = aderdg_last_error();
        s->eng.release();
        if (s->own_stream) cudaStreamDestroy(st);
        delete s;
        return fail(rc, m);
    }
    s->worker = std::thread([s] { s->loop(); });
    *out = s;
    return ADERDG_OK;
}

int aderdg_server_destroy(aderdg_server_t *s)
{
    if (!s) return ADERDG_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    cudaStream_t st = s->eng.st;
    s->eng.release();
    if (s->own_stream && st) cudaStreamDestroy(st);
    for (auto &kv : s->tickets) delete kv.second;
    delete s;
    return ADERDG_OK;
}

int aderdg_submit(aderdg_server_t *s, const aderdg_request_t *req, uint64_t *ticket)
{
    if (!s || !req || !ticket || !req->u0) return fail(ADERDG_E_INVAL, "NULL argument");
    if (!(req->t_end > 0) || !std::isfinite(req->t_end)) return fail(ADERDG_E_INVAL, "t_end must be positive");
    Request *r = new Request();
    const int prec = req->precision < 0 ? s->prec : req->precision;
    const int guess = req->initial_guess < 0 ? s->guess : req->initial_guess;
    if (prec != ADERDG_FP64 && prec != ADERDG_MIXED_FP32) { delete r; return fail(ADERDG_E_INVAL, "bad precision"); }
    int rc = make_slot(req->spec, prec, guess, 0, 0.0, r->spec);
    if (rc) { delete r; return rc; }
    if (r->spec.bytes > s->budget) {
        delete r;
        return fail(ADERDG_E_NOMEM, "request needs more device memory than the server budget");
    }
    const size_t nv = (size_t)r->spec.E * r->spec.NS * r->spec.M;
    r->u0.assign(req->u0, req->u0 + nv);
    r->t_end = req->t_end;
    r->submitted = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if ((int)s->queue.size() >= s->max_queue) {
            delete r;
            return fail(ADERDG_E_BUSY, "request queue is full");
        }
        r->ticket = s->next_ticket++;
        s->tickets[r->ticket] = r;
        s->queue.push_back(r);
        *ticket = r->ticket;
    }
    s->cv.notify_all();
    return ADERDG_OK;
}

int aderdg_poll(aderdg_server_t *s, uint64_t ticket, aderdg_result_t *res)
{
    if (!s || !res) return fail(ADERDG_E_INVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return fail(ADERDG_E_INVAL, "unknown ticket");
    Request *r = it->second;
    std::memset(res, 0, sizeof(*res));
    res->status = r->status;
    if (r->status == ADERDG_PENDING) return ADERDG_PENDING;
    res->latency_s = std::chrono::duration<double>(r->finished - r->submitted).count();
    res->queue_s = r->admitted.time_since_epoch().count()
                       ? std::chrono::duration<double>(r->admitted - r->submitted).count() : res->latency_s;
    res->t = r->t;
    res->steps = r->steps;
    res->u = r->result.empty() ? nullptr : r->result.data();
    res->n_values = r->result.size();
    if (r->status < 0) return fail(r->status, "request failed");
    return ADERDG_OK;
}

int aderdg_release(aderdg_server_t *s, uint64_t ticket)
{
    if (!s) return fail(ADERDG_E_INVAL, "NULL server");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return fail(ADERDG_E_INVAL, "unknown ticket");
    if (it->second->status == ADERDG_PENDING) return fail(ADERDG_E_BUSY, "request still running; cancel it first");
    delete it->second;
    s->tickets.erase(it);
    return ADERDG_OK;
}

int aderdg_cancel(aderdg_server_t *s, uint64_t ticket)
{
    if (!s) return fail(ADERDG_E_INVAL, "NULL server");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return fail(ADERDG_E_INVAL, "unknown ticket");
    it->second->cancelled = true;
    return ADERDG_OK;
}

int aderdg_server_stats(aderdg_server_t *s, int64_t *queued, int64_t *active, int64_t *finished,
                        size_t *bytes_in_use)
{
    if (!s) return fail(ADERDG_E_INVAL, "NULL server");
    std::lock_guard<std::mutex> lk(s->mu);
    if (queued) *queued = (int64_t)s->queue.size();
    if (active) *active = (int64_t)s->running.size();
    if (finished) *finished = s->finished;
    if (bytes_in_use) *bytes_in_use = s->eng.mem.in_use;
    return ADERDG_OK;
}

}  // extern "C"
