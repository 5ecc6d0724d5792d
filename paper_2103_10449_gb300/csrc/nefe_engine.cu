// libnefe engine: a context holding many systems (replicas of uneven size, dCCI pairs)
// that advance together; every step is the kernel sequence of nefe_kernels.cu, and runs
// of many steps replay a captured CUDA graph of kGraphSteps steps.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "nefe.h"
#include "nefe_dev.h"
#include "nefe_host.h"
#include "nefe_launch.h"
#include "nefe_nvtx.h"

using namespace nefe;

namespace {

constexpr int kGraphSteps = 32;

struct HostSys {
    int n = 0;
    std::vector<double> x, v, r0;
    double box[3] = {0, 0, 0};
    double mass = 28.0855;
    int pot = NEFE_POT_SW;
    double k_int = 0.0;
    nefe_sw_params prm{};
    nefe_uf_params uf{25.0, 2.0, 2200.0, 8.0};
    double T = 0.0, tdamp = 0.0;
    uint64_t seed = 0;
    int baro = NEFE_BARO_NONE;
    double P_GPa = 0.0, pdamp = 1.0;
    nefe_schedule sched{};
    int pair = -1;
    int trace_every = 0;
    long trace_cap = 0;
};

struct HostPair {
    int a, b, mode;
    double T0, P0, frm, to;
    long nsteps;
};

}  // namespace

struct nefe_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int prec = NEFE_FP32;
    double dt = 0.001, skin = 0.5;
    int cap = 48;
    std::vector<HostSys> sys;
    std::vector<HostPair> pairs;
    bool ready = false;
    int ntot = 0, ntiles = 0, nsys = 0, ngroups = 0;
    long long ncells_total = 0, trace_total = 0;
    DevSys* d_sys = nullptr;
    DevState* d_st = nullptr;
    long long* d_acc = nullptr;
    long long* d_acc_tmp = nullptr;
    int* d_tile_sys = nullptr;
    double *d_x = nullptr, *d_r0 = nullptr, *d_ftmp = nullptr, *d_vtmp = nullptr;
    void *d_v = nullptr, *d_dhi = nullptr, *d_dlo = nullptr;
    void *d_F = nullptr, *d_xs = nullptr, *d_xa = nullptr, *d_xcs = nullptr, *d_sd0 = nullptr, *d_xi = nullptr;
    void *d_shd = nullptr, *d_P = nullptr, *d_spill = nullptr;
    int *d_shj = nullptr, *d_shn = nullptr, *d_rtiles = nullptr, *d_rcount = nullptr, *d_rcbase = nullptr;
    int* d_any = nullptr;    // context-wide rebuild flag words (Bufs::any_rebuild)
    int *d_uf_nbr = nullptr, *d_uf_cnt = nullptr, *d_uf_tiles = nullptr;
    int* d_lacc = nullptr;   // scatter-form force accumulators (FP32 contexts)
    void* d_uf_F = nullptr;
    int n_uf_tiles = 0;      // tiles of the systems with a Uhlenbeck-Ford term
    int4* d_q = nullptr;
    int *d_cell_of = nullptr, *d_perm = nullptr, *d_cell_start = nullptr, *d_cell_count = nullptr,
        *d_cell_cursor = nullptr, *d_nbr = nullptr, *d_cnt = nullptr;
    void* d_swc = nullptr;
    DevPair* d_pairs = nullptr;
    DevGroup* d_groups = nullptr;
    double* d_trace = nullptr;
    std::vector<void*> allocs;
    int lanes = 8;           // pass A lanes per atom (1 = one thread per atom, 4, 8, 16, 32; 0 = one
                             // thread per atom in the scatter form, whose pass B is k_finish)
    int glanes = 4;          // pass B lanes per atom (1, 2, 4, 8)
    int llanes = 0;          // list build: 0 one warp per cell; 8, 16, 32 lanes per atom
    int rebuild_all = 0;     // rebuild policy (nefe_set_rebuild_policy)
    double tune_us = 0.0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    long launches = 0;
    long graph_launches = 0;     // kernel launches in one replay of the captured graph
    bool any_baro = false;       // some system has a barostat (k_kick_drift has work every step)
    int coop_blocks = 0;         // grid of the single-launch rebuild (0: cannot be launched)
    bool coop = false;           // rebuild as one cooperative launch (nefe_set_cooperative_rebuild)
    bool profiling = false;
    std::vector<cudaEvent_t> ev0, ev1, ev2;   // around the force passes of the captured graph
    std::vector<int> chunk_tile0, chunk_ntile;
    // force passes run over whole systems of at most this many atoms per launch (one launch:
    // splitting into L2-sized chunks was measured no faster once pass B only gathers leg forces)
    int chunk_atoms = 1 << 30;
    std::vector<int> sys_tile0, sys_n;
    int ntiles_total = 0;
    Bufs b{};
};

namespace {

// Groups whole systems into chunks of at most `atoms` atoms (a larger system is a chunk of
// its own).
void plan_chunks(nefe_ctx* c, int atoms_max) {
    c->chunk_atoms = atoms_max;
    c->chunk_tile0.clear();
    c->chunk_ntile.clear();
    int t0 = 0, atoms = 0;
    for (size_t s = 0; s < c->sys_n.size(); ++s) {
        if (atoms > 0 && (long long)atoms + c->sys_n[s] > atoms_max) {
            c->chunk_tile0.push_back(t0);
            c->chunk_ntile.push_back(c->sys_tile0[s] - t0);
            t0 = c->sys_tile0[s];
            atoms = 0;
        }
        atoms += c->sys_n[s];
    }
    c->chunk_tile0.push_back(t0);
    c->chunk_ntile.push_back(c->ntiles_total - t0);
}

int set_device(nefe_ctx* c) {
    NEFE_CU(cudaSetDevice(c->device));
    return NEFE_OK;
}

template <typename P>
int dalloc(nefe_ctx* c, P** p, size_t bytes) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, bytes < 16 ? 16 : bytes);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
    c->allocs.push_back(q);
    *p = static_cast<P*>(q);
    return NEFE_OK;
}

int check_sys(nefe_ctx* c, int s) {
    if (!c) return fail(NEFE_EINVAL, "context is NULL");
    if (s < 0 || s >= (int)c->sys.size()) return fail(NEFE_EINVAL, "system %d does not exist", s);
    return NEFE_OK;
}

int not_ready(nefe_ctx* c, const char* what) {
    if (c->ready) return fail(NEFE_ESTATE, "%s: only allowed before nefe_setup / nefe_run", what);
    return NEFE_OK;
}

double rc_of(const HostSys& h) { return h.prm.a * h.prm.sigma; }

// Both force passes, chunk by chunk; with slot >= 0 (profiling capture) events bracket
// every chunk's pass A and pass B.  fuse: the scatter form's epilogue also runs the next
// step's kick and drift for the systems without a barostat.
void enqueue_forces(nefe_ctx* c, int mode, int slot = -1, int fuse = 0) {
    if (c->n_uf_tiles > 0) launch_uf(c->b, c->prec, c->n_uf_tiles, mode, c->stream, &c->launches);
    const int nch = (int)c->chunk_tile0.size();
    for (int k = 0; k < nch; ++k) {
        Bufs b = c->b;
        b.tile_base = c->chunk_tile0[k];
        const int e = slot >= 0 ? slot * nch + k : -1;
        const bool prof = e >= 0 && e < (int)c->ev0.size();
        if (prof) cudaEventRecordWithFlags(c->ev0[e], c->stream, cudaEventRecordExternal);
        launch_edges(b, c->prec, c->lanes, c->chunk_ntile[k], mode, c->stream, &c->launches);
        if (prof) cudaEventRecordWithFlags(c->ev1[e], c->stream, cudaEventRecordExternal);
        launch_gather(b, c->prec, c->lanes == 0 ? 0 : c->glanes, c->chunk_ntile[k], mode, c->stream, &c->launches,
                      fuse);
        if (prof) cudaEventRecordWithFlags(c->ev2[e], c->stream, cudaEventRecordExternal);
    }
}

// One MD step.  first / last: the step's place in a sequence enqueued together (a captured
// graph, or the steps left over after the graph replays).  In the scatter form, every step but
// the last hands the next step's kick and drift of the systems without a barostat to its own
// epilogue (k_finish), so that the next step's k_kick_drift skips them; the last step of a
// sequence does not, so between calls the state is at a full step as usual.
void enqueue_step(nefe_ctx* c, int slot = -1, bool first = true, bool last = true) {
    NvtxRange nvtx_("nefe step");
    const bool fused = c->lanes == 0;            // k_finish is the epilogue
    launch_group(c->b, c->d_groups, c->ngroups, 1, c->stream, &c->launches, fused && !first);
    // with every system moved by the previous epilogue there is nothing left for k_kick_drift
    if (!(fused && !first && !c->any_baro))
        launch_kick_drift(c->b, c->prec, c->ntiles, 1, c->stream, &c->launches, fused && !first);
    // the rebuild: one cooperative launch (worklist, cells, lists between grid barriers), or the
    // kernel sequence where the list build has lanes per atom or UF rows are built too
    if (c->coop && c->coop_blocks > 0 && c->llanes == 0 && c->n_uf_tiles == 0) {
        launch_rebuild_coop(c->b, c->prec, c->coop_blocks, c->nsys, c->stream, &c->launches);
    } else {
        launch_cells_and_list(c->b, c->prec, c->ntiles, c->nsys, 0, c->stream, &c->launches);
        if (c->n_uf_tiles > 0) launch_uf_list(c->b, c->prec, c->ntiles, c->stream, &c->launches);
    }
    enqueue_forces(c, FM_STEP, slot, fused && !last);
}

void fill_results(const DevSys& S, const DevState& st, nefe_results* out) {
    std::memset(out, 0, sizeof(*out));
    out->W = st.W;
    out->lambda = S.sched == NEFE_SCHED_AS ? st.lam * kEvA3ToGPa : st.lam;
    out->step = (long)st.k;
    out->U = st.u_int;
    out->U_E = st.u_ref;
    out->K = 0.5 * (st.kt[0] + st.kt[1] + st.kt[2]);
    out->T = (st.kt[0] + st.kt[1] + st.kt[2]) / ((3.0 * S.n - 3.0) * kB);
    for (int k = 0; k < 6; ++k) out->P[k] = st.P[k] * kEvA3ToGPa;
    out->V = st.V;
    for (int k = 0; k < 3; ++k) out->box[k] = st.box[k];
    out->dHdl = st.dHdl;
    out->H = st.H;
    const double cnt = st.sums[4] > 0 ? st.sums[4] : 1.0;
    out->mean_H = st.sums[0] / cnt;
    out->mean_dHdl = st.sums[1] / cnt;
    out->mean_P = st.sums[2] / cnt * kEvA3ToGPa;
    out->mean_V = st.sums[3] / cnt;
    double pt;
    if (S.sched == NEFE_SCHED_RS) pt = st.lam * S.p_phys;
    else if (S.sched == NEFE_SCHED_AS) pt = st.lam;
    else if (S.pair >= 0) pt = st.p_tgt;
    else pt = S.p_ext;
    out->P_target = pt * kEvA3ToGPa;
    out->error = st.err;
}

// Lists, mirror and total forces from the current x, v (lambda and scales unchanged).
int resetup(nefe_ctx* c) {
    NEFE_CU(cudaMemsetAsync(c->d_acc, 0, sizeof(long long) * (size_t)c->nsys * ACC_N * kSlots, c->stream));
    if (c->d_lacc) NEFE_CU(cudaMemsetAsync(c->d_lacc, 0, 4 * sizeof(int) * (size_t)c->ntot, c->stream));
    launch_cells_and_list(c->b, c->prec, c->ntiles, c->nsys, 1, c->stream, &c->launches);
    if (c->n_uf_tiles > 0) launch_uf_list(c->b, c->prec, c->ntiles, c->stream, &c->launches);
    launch_kick_drift(c->b, c->prec, c->ntiles, 0, c->stream, &c->launches);
    enqueue_forces(c, FM_SETUP);
    NEFE_CU(cudaGetLastError());
    return NEFE_OK;
}

// Event slots for profiling: three per chunk per captured step.
int ensure_events(nefe_ctx* c) {
    const size_t ne = (size_t)kGraphSteps * std::max<size_t>(1, c->chunk_tile0.size());
    if (c->ev0.size() == ne) return NEFE_OK;
    for (auto e : c->ev0) cudaEventDestroy(e);
    for (auto e : c->ev1) cudaEventDestroy(e);
    for (auto e : c->ev2) cudaEventDestroy(e);
    c->ev0.assign(ne, nullptr);
    c->ev1.assign(ne, nullptr);
    c->ev2.assign(ne, nullptr);
    for (size_t k = 0; k < ne; ++k) {
        NEFE_CU(cudaEventCreate(&c->ev0[k]));
        NEFE_CU(cudaEventCreate(&c->ev1[k]));
        NEFE_CU(cudaEventCreate(&c->ev2[k]));
    }
    return NEFE_OK;
}

void drop_graph(nefe_ctx* c) {
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->graph) cudaGraphDestroy(c->graph);
    c->gexec = nullptr;
    c->graph = nullptr;
}

int setup(nefe_ctx* c) {
    if (c->ready) return NEFE_OK;
    if (c->sys.empty()) return fail(NEFE_ESTATE, "nefe_setup: no systems");
    int rc = set_device(c);
    if (rc) return rc;
    const int nsys = (int)c->sys.size();
    std::vector<DevSys> hs(nsys);
    std::vector<DevState> hst(nsys);
    std::vector<int> tile_sys;
    long long ntot = 0, ncell = 0, tr = 0;
    for (int s = 0; s < nsys; ++s) {
        HostSys& h = c->sys[s];
        const double rcs = rc_of(h) + c->skin;
        int n3[3];
        if (!host_grid(h.box, rcs, n3))
            return fail(NEFE_EINVAL, "system %d: box below 2 (rc + skin) = %g", s, 2 * rcs);
        // room for the box to grow by 25 % per axis under a barostat
        long long cap = 1;
        for (int k = 0; k < 3; ++k) cap *= (long long)std::max(2, (int)std::floor(n3[k] * 1.25) + 1);
        DevSys& d = hs[s];
        std::memset(&d, 0, sizeof(d));
        d.off = (int)ntot;
        d.n = h.n;
        d.tile0 = (int)tile_sys.size();
        d.ntile = (h.n + kTile - 1) / kTile;
        for (int t = 0; t < d.ntile; ++t) tile_sys.push_back(s);
        d.cell0 = (int)ncell;
        d.ncell_cap = (int)cap;
        d.pot = h.pot;
        d.sched = h.sched.kind;
        d.direction = h.sched.direction < 0 ? -1 : 1;
        d.nsched = h.sched.nsteps > 0 ? h.sched.nsteps : 1;
        d.k_int = h.k_int;
        const bool uf_ref = h.sched.kind == NEFE_SCHED_FL && h.sched.ref == NEFE_REF_UF;
        d.k_E = (h.sched.kind == NEFE_SCHED_FL && !uf_ref) ? h.sched.k_E : 0.0;
        d.uf_mode = h.pot == NEFE_POT_UF ? UF_INT : (uf_ref ? UF_REF : UF_NONE);
        if (h.pot == NEFE_POT_UF && uf_ref)
            return fail(NEFE_EINVAL, "system %d: the UF fluid cannot be its own FL reference", s);
        if (d.uf_mode != UF_NONE) {
            fill_uf(d, h.uf, c->skin, d.uf_mode);
            const double R = h.uf.rc + c->skin;
            if (R > 2.0 * rcs)
                return fail(NEFE_EINVAL, "system %d: UF rc + skin = %g above 2 (a sigma + skin) = %g", s, R, 2.0 * rcs);
            for (int k = 0; k < 3; ++k) {
                if (h.box[k] < 2.0 * R)
                    return fail(NEFE_EINVAL, "system %d: box %g below 2 (UF rc + skin) = %g", s, h.box[k], 2.0 * R);
                if (n3[k] < 5) return fail(NEFE_EINVAL, "system %d: a UF system needs >= 5 cells per axis", s);
            }
        }
        d.lam_f = h.sched.lambda_f;
        d.p_phys = h.sched.P_GPa / kEvA3ToGPa;
        d.p0 = h.sched.P0_GPa / kEvA3ToGPa;
        d.p1 = h.sched.P1_GPa / kEvA3ToGPa;
        d.lam0 = h.sched.kind == NEFE_SCHED_NONE ? h.sched.lambda0 : 1.0;
        d.mass_e = h.mass * kMvv2e;
        d.T = h.T;
        d.tdamp = h.tdamp;
        d.seed = h.seed;
        d.rng_id = s;
        d.pair = h.pair;
        d.baro = h.baro;
        if (h.baro != NEFE_BARO_NONE) c->any_baro = true;
        d.p_ext = h.P_GPa / kEvA3ToGPa;
        d.pdamp = h.pdamp;
        d.rcs = rcs;
        d.skin = c->skin;
        d.amp = h.tdamp > 0.0 ? std::sqrt(2.0 * d.mass_e * kB * h.T / (h.tdamp * c->dt)) : 0.0;
        d.gam = h.tdamp > 0.0 ? d.mass_e / h.tdamp : 0.0;
        d.ckick = 0.5 * c->dt / d.mass_e;
        d.amp_f = (float)d.amp; d.gam_f = (float)d.gam; d.ckick_f = (float)d.ckick;
        d.mass_f = (float)d.mass_e; d.kE_f = (float)d.k_E; d.kint_f = (float)d.k_int;
        d.dt_f = (float)c->dt;
        d.inv_n_f = (float)(1.0 / h.n);
        d.rcs2_lo_f = (float)(rcs * rcs) * (1.0f - 1e-4f);
        d.rcs2_hi_f = (float)(rcs * rcs) * (1.0f + 1e-4f);
        d.thermo = h.tdamp > 0.0 ? 1 : 0;
        d.springs = (d.k_E > 0.0 || h.pot == NEFE_POT_EINSTEIN) ? 1 : 0;
        d.trace_every = h.trace_every;
        d.trace_cap = h.trace_cap;
        d.trace_off = tr;
        d.prm = s;
        DevState& st = hst[s];
        std::memset(&st, 0, sizeof(st));
        for (int k = 0; k < 3; ++k) { st.box[k] = h.box[k]; st.s[k] = 1.0; st.phi[k] = 1.0; }
        st.lam = d.lam0;
        st.rebuild = 1;
        ntot += h.n;
        ncell += cap;
        tr += h.trace_every > 0 ? h.trace_cap : 0;
    }
    if (ntot >= (1LL << kCodeShift)) return fail(NEFE_EINVAL, "more than 2^27 atoms in one context");
    std::vector<int> uf_tiles;
    for (int s = 0; s < nsys; ++s)
        if (hs[s].uf_mode != UF_NONE)
            for (int t = 0; t < hs[s].ntile; ++t) uf_tiles.push_back(hs[s].tile0 + t);
    if (!uf_tiles.empty() && ntot >= (1LL << kUfShift))
        return fail(NEFE_EINVAL, "more than 2^25 atoms in a context with UF systems");
    c->sys_tile0.resize(nsys);
    c->sys_n.resize(nsys);
    for (int s = 0; s < nsys; ++s) { c->sys_tile0[s] = hs[s].tile0; c->sys_n[s] = hs[s].n; }
    c->ntiles_total = (int)tile_sys.size();
    plan_chunks(c, c->chunk_atoms);
    c->ntot = (int)ntot;
    c->ntiles = (int)tile_sys.size();
    c->nsys = nsys;
    c->ncells_total = ncell;
    c->trace_total = tr;
    // groups: each dCCI pair, then every system outside a pair
    std::vector<DevGroup> groups;
    std::vector<DevPair> hp(c->pairs.size());
    for (size_t p = 0; p < c->pairs.size(); ++p) {
        const HostPair& P = c->pairs[p];
        DevPair& d = hp[p];
        std::memset(&d, 0, sizeof(d));
        d.a = P.a; d.b = P.b; d.mode = P.mode; d.T0 = P.T0;
        const double conv = P.mode == NEFE_DCCI_PRESS ? 1.0 / kEvA3ToGPa : 1.0;
        d.frm = P.frm * conv; d.to = P.to * conv;
        d.nsteps = P.nsteps > 0 ? P.nsteps : 1;
        d.lam = 1.0;
        d.ps = P.P0 / kEvA3ToGPa;
        groups.push_back(DevGroup{P.a, P.b, (int)p, 0});
        hst[P.a].p_tgt = d.ps;
        hst[P.b].p_tgt = d.ps;
    }
    for (int s = 0; s < nsys; ++s)
        if (c->sys[s].pair < 0) groups.push_back(DevGroup{s, -1, -1, 0});
    c->ngroups = (int)groups.size();

    const size_t N = (size_t)ntot;
    const size_t v4 = c->prec == NEFE_FP64 ? sizeof(double4) : sizeof(float4);
    const size_t el = c->prec == NEFE_FP64 ? sizeof(double) : sizeof(float);
    if ((rc = dalloc(c, &c->d_sys, sizeof(DevSys) * nsys))) return rc;
    if ((rc = dalloc(c, &c->d_st, sizeof(DevState) * nsys))) return rc;
    if ((rc = dalloc(c, &c->d_acc, sizeof(long long) * nsys * ACC_N * kSlots))) return rc;
    if ((rc = dalloc(c, &c->d_acc_tmp, sizeof(long long) * nsys * ACC_N * kSlots))) return rc;
    if ((rc = dalloc(c, &c->d_tile_sys, sizeof(int) * tile_sys.size()))) return rc;
    if ((rc = dalloc(c, &c->d_x, sizeof(double) * 3 * N))) return rc;
    if ((rc = dalloc(c, &c->d_v, el * 3 * N))) return rc;
    if ((rc = dalloc(c, &c->d_dhi, el * 3 * N))) return rc;
    if ((rc = dalloc(c, &c->d_dlo, el * 3 * N))) return rc;
    if ((rc = dalloc(c, &c->d_r0, sizeof(double) * 3 * N))) return rc;
    if ((rc = dalloc(c, &c->d_ftmp, sizeof(double) * 3 * N))) return rc;
    if ((rc = dalloc(c, &c->d_vtmp, sizeof(double) * 3 * N))) return rc;
    if ((rc = dalloc(c, &c->d_F, v4 * N))) return rc;
    if ((rc = dalloc(c, &c->d_xs, v4 * N))) return rc;
    if ((rc = dalloc(c, &c->d_xa, v4 * N))) return rc;
    if ((rc = dalloc(c, &c->d_xcs, v4 * N))) return rc;
    if ((rc = dalloc(c, &c->d_sd0, v4 * N))) return rc;
    if ((rc = dalloc(c, &c->d_xi, v4 * N))) return rc;
    if ((rc = dalloc(c, &c->d_shd, v4 * N * (size_t)kShell))) return rc;
    // spill area of the thread-per-atom pass A (FP32 only): the last kSpill1 entries of a shell
    if (c->prec == NEFE_FP32 && (rc = dalloc(c, &c->d_spill, (v4 + sizeof(float)) * N * kSpill1))) return rc;
    if ((rc = dalloc(c, &c->d_shj, sizeof(int) * N * (size_t)kShell))) return rc;
    if ((rc = dalloc(c, &c->d_shn, sizeof(int) * N))) return rc;
    if ((rc = dalloc(c, &c->d_P, 3 * v4 * N))) return rc;
    if (c->prec == NEFE_FP32) {
        if ((rc = dalloc(c, &c->d_lacc, 4 * sizeof(int) * N))) return rc;
        NEFE_CU(cudaMemset(c->d_lacc, 0, 4 * sizeof(int) * N));
    }
    if ((rc = dalloc(c, &c->d_rtiles, sizeof(int) * tile_sys.size()))) return rc;
    if ((rc = dalloc(c, &c->d_rcount, sizeof(int)))) return rc;
    if ((rc = dalloc(c, &c->d_rcbase, sizeof(int) * (size_t)(nsys + 1)))) return rc;
    // [0], [1] rebuild flags of this and the next step, [2] barrier timeout, [3] barrier word
    if ((rc = dalloc(c, &c->d_any, sizeof(int) * 4))) return rc;
    NEFE_CU(cudaMemset(c->d_any, 0, sizeof(int) * 4));
    c->coop_blocks = rebuild_coop_blocks(c->prec);
    if ((rc = dalloc(c, &c->d_q, sizeof(int4) * N))) return rc;
    if ((rc = dalloc(c, &c->d_cell_of, sizeof(int) * N))) return rc;
    if ((rc = dalloc(c, &c->d_perm, sizeof(int) * N))) return rc;
    if ((rc = dalloc(c, &c->d_cell_start, sizeof(int) * (size_t)(ncell + nsys)))) return rc;
    if ((rc = dalloc(c, &c->d_cell_count, sizeof(int) * (size_t)ncell))) return rc;
    if ((rc = dalloc(c, &c->d_cell_cursor, sizeof(int) * (size_t)ncell))) return rc;
    if ((rc = dalloc(c, &c->d_nbr, sizeof(int) * N * (size_t)c->cap))) return rc;
    if ((rc = dalloc(c, &c->d_cnt, sizeof(int) * N))) return rc;
    if ((rc = dalloc(c, &c->d_pairs, sizeof(DevPair) * std::max<size_t>(1, hp.size())))) return rc;
    if ((rc = dalloc(c, &c->d_groups, sizeof(DevGroup) * groups.size()))) return rc;
    if ((rc = dalloc(c, &c->d_trace, sizeof(double) * 9 * (size_t)std::max<long long>(1, tr)))) return rc;
    c->n_uf_tiles = (int)uf_tiles.size();
    if (!uf_tiles.empty()) {
        if ((rc = dalloc(c, &c->d_uf_nbr, sizeof(int) * N * (size_t)kUfCap))) return rc;
        if ((rc = dalloc(c, &c->d_uf_cnt, sizeof(int) * N))) return rc;
        if ((rc = dalloc(c, &c->d_uf_F, v4 * N))) return rc;
        if ((rc = dalloc(c, &c->d_uf_tiles, sizeof(int) * uf_tiles.size()))) return rc;
        NEFE_CU(cudaMemcpy(c->d_uf_tiles, uf_tiles.data(), sizeof(int) * uf_tiles.size(), cudaMemcpyHostToDevice));
        NEFE_CU(cudaMemset(c->d_uf_cnt, 0, sizeof(int) * N));
        NEFE_CU(cudaMemset(c->d_uf_F, 0, v4 * N));
    }
    if (c->prec == NEFE_FP64) {
        std::vector<SWc<double>> t(nsys);
        for (int s = 0; s < nsys; ++s) t[s] = make_swc<double>(c->sys[s].prm);
        if ((rc = dalloc(c, &c->d_swc, sizeof(SWc<double>) * nsys))) return rc;
        NEFE_CU(cudaMemcpy(c->d_swc, t.data(), sizeof(SWc<double>) * nsys, cudaMemcpyHostToDevice));
    } else {
        std::vector<SWc<float>> t(nsys);
        for (int s = 0; s < nsys; ++s) t[s] = make_swc<float>(c->sys[s].prm);
        if ((rc = dalloc(c, &c->d_swc, sizeof(SWc<float>) * nsys))) return rc;
        NEFE_CU(cudaMemcpy(c->d_swc, t.data(), sizeof(SWc<float>) * nsys, cudaMemcpyHostToDevice));
    }
    // per-atom arrays: host (n,3) -> device SoA
    std::vector<double> hx(3 * N), hv(3 * N), hr(3 * N);
    for (int s = 0; s < nsys; ++s) {
        const HostSys& h = c->sys[s];
        const size_t off = hs[s].off;
        for (int i = 0; i < h.n; ++i)
            for (int k = 0; k < 3; ++k) {
                hx[k * N + off + i] = h.x[3 * i + k];
                hv[k * N + off + i] = h.v.empty() ? 0.0 : h.v[3 * i + k];
                hr[k * N + off + i] = h.r0.empty() ? h.x[3 * i + k] : h.r0[3 * i + k];
            }
    }
    NEFE_CU(cudaMemcpy(c->d_x, hx.data(), sizeof(double) * 3 * N, cudaMemcpyHostToDevice));
    NEFE_CU(cudaMemcpy(c->d_vtmp, hv.data(), sizeof(double) * 3 * N, cudaMemcpyHostToDevice));
    NEFE_CU(cudaMemcpy(c->d_r0, hr.data(), sizeof(double) * 3 * N, cudaMemcpyHostToDevice));
    NEFE_CU(cudaMemset(c->d_dhi, 0, el * 3 * N));
    NEFE_CU(cudaMemset(c->d_dlo, 0, el * 3 * N));
    NEFE_CU(cudaMemset(c->d_xi, 0, v4 * N));
    NEFE_CU(cudaMemcpy(c->d_sys, hs.data(), sizeof(DevSys) * nsys, cudaMemcpyHostToDevice));
    NEFE_CU(cudaMemcpy(c->d_st, hst.data(), sizeof(DevState) * nsys, cudaMemcpyHostToDevice));
    NEFE_CU(cudaMemcpy(c->d_tile_sys, tile_sys.data(), sizeof(int) * tile_sys.size(), cudaMemcpyHostToDevice));
    NEFE_CU(cudaMemcpy(c->d_groups, groups.data(), sizeof(DevGroup) * groups.size(), cudaMemcpyHostToDevice));
    if (!hp.empty())
        NEFE_CU(cudaMemcpy(c->d_pairs, hp.data(), sizeof(DevPair) * hp.size(), cudaMemcpyHostToDevice));
    NEFE_CU(cudaMemset(c->d_cell_count, 0, sizeof(int) * (size_t)ncell));
    NEFE_CU(cudaMemset(c->d_F, 0, v4 * N));
    NEFE_CU(cudaMemset(c->d_trace, 0, sizeof(double) * 9 * (size_t)std::max<long long>(1, tr)));

    Bufs& b = c->b;
    std::memset(&b, 0, sizeof(b));
    b.sys = c->d_sys; b.st = c->d_st; b.acc = c->d_acc; b.tile_sys = c->d_tile_sys;
    b.x = c->d_x; b.v = c->d_v; b.dhi = c->d_dhi; b.dlo = c->d_dlo; b.r0 = c->d_r0; b.F = c->d_F;
    b.xs = c->d_xs; b.xa = c->d_xa; b.xcs = c->d_xcs; b.sd0 = c->d_sd0; b.xi = c->d_xi;
    b.shd = c->d_shd; b.shj = c->d_shj; b.shn = c->d_shn; b.P = c->d_P; b.spill = c->d_spill;
    b.rtiles = c->d_rtiles; b.rcount = c->d_rcount; b.rcbase = c->d_rcbase; b.any_rebuild = c->d_any;
    b.q = c->d_q; b.cell_of = c->d_cell_of; b.perm = c->d_perm; b.cell_start = c->d_cell_start;
    b.cell_count = c->d_cell_count; b.cell_cursor = c->d_cell_cursor; b.nbr = c->d_nbr; b.cnt = c->d_cnt;
    b.cap = c->cap; b.ntot = c->ntot; b.dt = c->dt; b.swc = c->d_swc; b.pairs = c->d_pairs;
    b.nbr_il = (c->cap & 3) == 0 ? 1 : 0;   // interleaved rows (the force passes read them 4 at a time)
    b.rebuild_all = c->rebuild_all;

    b.trace = c->d_trace;
    b.list_lanes = c->llanes;
    b.uf_nbr = c->d_uf_nbr; b.uf_cnt = c->d_uf_cnt; b.uf_F = c->d_uf_F; b.uf_tiles = c->d_uf_tiles;
    b.lacc = c->d_lacc;

    launch_inject(b, c->prec, c->ntiles, nullptr, c->d_vtmp, c->stream);
    NEFE_CU(cudaMemsetAsync(c->d_acc, 0, sizeof(long long) * nsys * ACC_N * kSlots, c->stream));
    launch_group(b, c->d_groups, c->ngroups, 0, c->stream, &c->launches);
    c->ready = true;
    rc = resetup(c);
    if (rc) return rc;
    NEFE_CU(cudaStreamSynchronize(c->stream));
    return NEFE_OK;
}

}  // namespace

extern "C" {

int nefe_create(nefe_ctx** out, int device, void* stream, int precision, double dt_ps, double skin,
                int nbr_cap) {
    if (!out) return fail(NEFE_EINVAL, "out is NULL");
    *out = nullptr;
    if (precision != NEFE_FP32 && precision != NEFE_FP64) return fail(NEFE_EINVAL, "bad precision");
    if (!(dt_ps > 0.0) || !(skin > 0.0)) return fail(NEFE_EINVAL, "dt and skin must be positive");
    if (nbr_cap < 16 || nbr_cap > kMaxCap) return fail(NEFE_EINVAL, "nbr_cap must be in 16..64");
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return fail(NEFE_ECUDA, "no CUDA device available");
    }
    if (device < 0 || device >= ndev) return fail(NEFE_EINVAL, "device %d out of range", device);
    nefe_ctx* c = new nefe_ctx();
    c->device = device;
    c->prec = precision;
    c->dt = dt_ps;
    c->skin = skin;
    c->cap = nbr_cap;
    if (cudaSetDevice(device) != cudaSuccess) { delete c; return fail(NEFE_ECUDA, "cudaSetDevice failed"); }
    if (stream) {
        c->stream = (cudaStream_t)stream;
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete c;
            return fail(NEFE_ECUDA, "cudaStreamCreate failed");
        }
        c->own_stream = true;
    }
    *out = c;
    return NEFE_OK;
}

int nefe_destroy(nefe_ctx* c) {
    if (!c) return NEFE_OK;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    drop_graph(c);
    for (auto e : c->ev0) cudaEventDestroy(e);
    for (auto e : c->ev1) cudaEventDestroy(e);
    for (auto e : c->ev2) cudaEventDestroy(e);
    for (void* p : c->allocs) cudaFree(p);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
    return NEFE_OK;
}

int nefe_add_system(nefe_ctx* c, const nefe_system_desc* d, int* sys_id) {
    if (!c || !d) return fail(NEFE_EINVAL, "NULL argument");
    int rc = not_ready(c, "nefe_add_system");
    if (rc) return rc;
    if (d->n < 2 || !d->x) return fail(NEFE_EINVAL, "a system needs n >= 2 and positions");
    if (!(d->mass > 0.0)) return fail(NEFE_EINVAL, "mass must be positive");
    if (d->pot != NEFE_POT_SW && d->pot != NEFE_POT_EINSTEIN && d->pot != NEFE_POT_UF)
        return fail(NEFE_EINVAL, "bad pot");
    for (int k = 0; k < 3; ++k)
        if (!(d->box[k] > 0.0)) return fail(NEFE_EINVAL, "box must be positive");
    HostSys h;
    h.n = d->n;
    h.x.assign(d->x, d->x + 3 * (size_t)d->n);
    if (d->v) h.v.assign(d->v, d->v + 3 * (size_t)d->n);
    if (d->r0) h.r0.assign(d->r0, d->r0 + 3 * (size_t)d->n);
    for (int k = 0; k < 3; ++k) h.box[k] = d->box[k];
    h.mass = d->mass;
    h.pot = d->pot;
    h.k_int = d->k_int;
    nefe_sw_params_silicon(&h.prm);
    h.sched.kind = NEFE_SCHED_NONE;
    h.sched.direction = 1;
    h.sched.nsteps = 1;
    h.sched.lambda0 = 1.0;
    c->sys.push_back(h);
    if (sys_id) *sys_id = (int)c->sys.size() - 1;
    return NEFE_OK;
}

int nefe_set_sw_params(nefe_ctx* c, int s, const nefe_sw_params* p) {
    if (!c) return fail(NEFE_EINVAL, "context is NULL");
    int rc = not_ready(c, "nefe_set_sw_params");
    if (rc) return rc;
    if (!valid_params(p)) return fail(NEFE_EINVAL, "invalid SW parameters");
    if (s == -1) {
        for (auto& h : c->sys) h.prm = *p;
        return NEFE_OK;
    }
    if ((rc = check_sys(c, s))) return rc;
    c->sys[s].prm = *p;
    return NEFE_OK;
}

int nefe_set_uf_params(nefe_ctx* c, int s, const nefe_uf_params* uf) {
    int rc = check_sys(c, s);
    if (rc) return rc;
    if ((rc = not_ready(c, "nefe_set_uf_params"))) return rc;
    if (!valid_uf(uf)) return fail(NEFE_EINVAL, "UF parameters must be positive and finite");
    c->sys[s].uf = *uf;
    return NEFE_OK;
}

int nefe_set_thermostat(nefe_ctx* c, int s, double T, double damp, uint64_t seed) {
    int rc = check_sys(c, s);
    if (rc) return rc;
    if ((rc = not_ready(c, "nefe_set_thermostat"))) return rc;
    if (!(T >= 0.0)) return fail(NEFE_EINVAL, "T must be >= 0");
    c->sys[s].T = T;
    c->sys[s].tdamp = damp > 0.0 ? damp : 0.0;
    c->sys[s].seed = seed;
    return NEFE_OK;
}

int nefe_set_barostat(nefe_ctx* c, int s, int mode, double P, double pdamp) {
    int rc = check_sys(c, s);
    if (rc) return rc;
    if ((rc = not_ready(c, "nefe_set_barostat"))) return rc;
    if (mode < NEFE_BARO_NONE || mode > NEFE_BARO_ANISO) return fail(NEFE_EINVAL, "bad barostat mode");
    if (mode != NEFE_BARO_NONE && !(pdamp > 0.0)) return fail(NEFE_EINVAL, "pdamp must be positive");
    c->sys[s].baro = mode;
    c->sys[s].P_GPa = P;
    c->sys[s].pdamp = pdamp;
    return NEFE_OK;
}

int nefe_set_schedule(nefe_ctx* c, int s, const nefe_schedule* sc) {
    int rc = check_sys(c, s);
    if (rc) return rc;
    if ((rc = not_ready(c, "nefe_set_schedule"))) return rc;
    if (!sc || sc->kind < NEFE_SCHED_NONE || sc->kind > NEFE_SCHED_AS) return fail(NEFE_EINVAL, "bad schedule");
    if (sc->kind != NEFE_SCHED_NONE && sc->nsteps < 1) return fail(NEFE_EINVAL, "schedule nsteps must be >= 1");
    if (sc->kind == NEFE_SCHED_RS && !(sc->lambda_f > 0.0)) return fail(NEFE_EINVAL, "lambda_f must be > 0");
    if (sc->kind == NEFE_SCHED_FL && sc->ref != NEFE_REF_EINSTEIN && sc->ref != NEFE_REF_UF)
        return fail(NEFE_EINVAL, "bad FL reference");
    if (sc->kind == NEFE_SCHED_FL && sc->ref == NEFE_REF_EINSTEIN && !(sc->k_E > 0.0))
        return fail(NEFE_EINVAL, "k_E must be > 0");
    if (c->sys[s].pair >= 0 && sc->kind != NEFE_SCHED_NONE)
        return fail(NEFE_EINVAL, "systems of a dCCI pair take no schedule");
    c->sys[s].sched = *sc;
    if (c->sys[s].sched.direction == 0) c->sys[s].sched.direction = 1;
    return NEFE_OK;
}

int nefe_pair_dcci(nefe_ctx* c, int a, int b, double T0, double P0, int mode, double frm, double to,
                   long nsteps, int* pair_id) {
    int rc = check_sys(c, a);
    if (rc) return rc;
    if ((rc = check_sys(c, b))) return rc;
    if ((rc = not_ready(c, "nefe_pair_dcci"))) return rc;
    if (a == b) return fail(NEFE_EINVAL, "a pair needs two different systems");
    if (c->sys[a].pair >= 0 || c->sys[b].pair >= 0) return fail(NEFE_EINVAL, "system already paired");
    if (mode != NEFE_DCCI_TEMP && mode != NEFE_DCCI_PRESS) return fail(NEFE_EINVAL, "bad dCCI mode");
    if (nsteps < 1 || !(T0 > 0.0)) return fail(NEFE_EINVAL, "bad nsteps or T0");
    if (mode == NEFE_DCCI_TEMP && (frm != T0 || !(to > 0.0)))
        return fail(NEFE_EINVAL, "temperature control starts at T0 and needs to > 0");
    if (c->sys[a].baro == NEFE_BARO_NONE || c->sys[b].baro == NEFE_BARO_NONE)
        return fail(NEFE_EINVAL, "both systems of a dCCI pair need a barostat");
    HostPair p{a, b, mode, T0, P0, frm, to, nsteps};
    c->pairs.push_back(p);
    const int id = (int)c->pairs.size() - 1;
    for (int s : {a, b}) {
        c->sys[s].pair = id;
        c->sys[s].T = T0;
        c->sys[s].sched.kind = NEFE_SCHED_NONE;
        c->sys[s].sched.lambda0 = 1.0;
    }
    if (pair_id) *pair_id = id;
    return NEFE_OK;
}

int nefe_set_trace(nefe_ctx* c, int s, int every, long cap) {
    int rc = check_sys(c, s);
    if (rc) return rc;
    if ((rc = not_ready(c, "nefe_set_trace"))) return rc;
    if (every < 0 || cap < 0) return fail(NEFE_EINVAL, "bad trace settings");
    c->sys[s].trace_every = every;
    c->sys[s].trace_cap = cap;
    return NEFE_OK;
}

int nefe_setup(nefe_ctx* c) {
    NvtxRange nvtx_("nefe_setup");
    if (!c) return fail(NEFE_EINVAL, "context is NULL");
    return setup(c);
}

int nefe_run(nefe_ctx* c, long nsteps) {
    NvtxRange nvtx_("nefe_run");
    if (!c) return fail(NEFE_EINVAL, "context is NULL");
    if (nsteps < 0) return fail(NEFE_EINVAL, "nsteps < 0");
    int rc = setup(c);
    if (rc) return rc;
    if ((rc = set_device(c))) return rc;
    long full = nsteps / kGraphSteps, rem = nsteps % kGraphSteps;
    if (full > 0 && !c->gexec) {
        if (c->profiling && (rc = ensure_events(c))) return rc;
        NEFE_CU(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
        long before = c->launches;
        for (int k = 0; k < kGraphSteps; ++k)
            enqueue_step(c, c->profiling ? k : -1, k == 0, k == kGraphSteps - 1);
        c->graph_launches = c->launches - before;
        c->launches = before;
        cudaError_t e = cudaStreamEndCapture(c->stream, &c->graph);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&c->gexec, c->graph, 0);
        if (e != cudaSuccess) { drop_graph(c); return cuda_fail(e, "cudaGraphInstantiate"); }
    }
    for (long f = 0; f < full; ++f) {
        NEFE_CU(cudaGraphLaunch(c->gexec, c->stream));
        c->launches += c->graph_launches;
    }
    for (long r = 0; r < rem; ++r) enqueue_step(c, -1, r == 0, r == rem - 1);
    NEFE_CU(cudaGetLastError());
    return NEFE_OK;
}

int nefe_sync(nefe_ctx* c) {
    if (!c) return fail(NEFE_EINVAL, "context is NULL");
    int rc = set_device(c);
    if (rc) return rc;
    NEFE_CU(cudaStreamSynchronize(c->stream));
    if (c->d_any) {
        int w[2] = {0, 0};
        NEFE_CU(cudaMemcpy(w, c->d_any + 2, sizeof(w), cudaMemcpyDeviceToHost));
        if (w[0]) {
            NEFE_CU(cudaMemset(c->d_any + 2, 0, 2 * sizeof(int)));   // the barrier starts afresh
            return fail(NEFE_ETIMEOUT, "a grid barrier of the list rebuild gave up waiting");
        }
    }
    return NEFE_OK;
}

int nefe_get_results(nefe_ctx* c, int s, nefe_results* out) {
    int rc = check_sys(c, s);
    if (rc) return rc;
    if (!out) return fail(NEFE_EINVAL, "out is NULL");
    if ((rc = setup(c))) return rc;
    if ((rc = set_device(c))) return rc;
    launch_group(c->b, c->d_groups, c->ngroups, 2, c->stream, &c->launches);
    DevState st;
    DevSys S;
    NEFE_CU(cudaMemcpyAsync(&st, c->d_st + s, sizeof(st), cudaMemcpyDeviceToHost, c->stream));
    NEFE_CU(cudaMemcpyAsync(&S, c->d_sys + s, sizeof(S), cudaMemcpyDeviceToHost, c->stream));
    NEFE_CU(cudaStreamSynchronize(c->stream));
    fill_results(S, st, out);
    return NEFE_OK;
}

int nefe_get_pair(nefe_ctx* c, int p, double* T_coex, double* P_coex, double* lambda, unsigned* error) {
    if (!c) return fail(NEFE_EINVAL, "context is NULL");
    if (p < 0 || p >= (int)c->pairs.size()) return fail(NEFE_EINVAL, "pair %d does not exist", p);
    int rc = setup(c);
    if (rc) return rc;
    if ((rc = set_device(c))) return rc;
    DevPair d;
    NEFE_CU(cudaMemcpyAsync(&d, c->d_pairs + p, sizeof(d), cudaMemcpyDeviceToHost, c->stream));
    NEFE_CU(cudaStreamSynchronize(c->stream));
    if (T_coex) *T_coex = d.T0 / d.lam;
    if (P_coex) *P_coex = d.ps / d.lam * kEvA3ToGPa;
    if (lambda) *lambda = d.lam;
    if (error) *error = d.err;
    return NEFE_OK;
}

int nefe_get_state(nefe_ctx* c, int s, double* x, double* v, double* box) {
    NvtxRange nvtx_("nefe_get_state");
    int rc = check_sys(c, s);
    if (rc) return rc;
    if ((rc = setup(c))) return rc;
    if ((rc = set_device(c))) return rc;
    const int n = c->sys[s].n;
    DevSys S;
    NEFE_CU(cudaMemcpyAsync(&S, c->d_sys + s, sizeof(S), cudaMemcpyDeviceToHost, c->stream));
    launch_materialize(c->b, c->prec, c->ntiles, c->d_ftmp, c->d_vtmp, c->stream);
    NEFE_CU(cudaStreamSynchronize(c->stream));
    std::vector<double> tmp(3 * (size_t)n);
    const size_t N = c->ntot;
    for (int which = 0; which < 2; ++which) {
        double* dst = which == 0 ? x : v;
        const double* src = which == 0 ? c->d_ftmp : c->d_vtmp;
        if (!dst) continue;
        for (int k = 0; k < 3; ++k)
            NEFE_CU(cudaMemcpyAsync(tmp.data() + (size_t)k * n, src + k * N + S.off, sizeof(double) * n,
                                    cudaMemcpyDeviceToHost, c->stream));
        NEFE_CU(cudaStreamSynchronize(c->stream));
        for (int i = 0; i < n; ++i)
            for (int k = 0; k < 3; ++k) dst[3 * i + k] = tmp[(size_t)k * n + i];
    }
    if (box) {
        DevState st;
        NEFE_CU(cudaMemcpyAsync(&st, c->d_st + s, sizeof(st), cudaMemcpyDeviceToHost, c->stream));
        NEFE_CU(cudaStreamSynchronize(c->stream));
        for (int k = 0; k < 3; ++k) box[k] = st.box[k];
    }
    return NEFE_OK;
}

int nefe_set_state(nefe_ctx* c, int s, const double* x, const double* v) {
    NvtxRange nvtx_("nefe_set_state");
    int rc = check_sys(c, s);
    if (rc) return rc;
    if ((rc = setup(c))) return rc;
    if ((rc = set_device(c))) return rc;
    const int n = c->sys[s].n;
    const size_t N = c->ntot;
    DevSys S;
    NEFE_CU(cudaMemcpyAsync(&S, c->d_sys + s, sizeof(S), cudaMemcpyDeviceToHost, c->stream));
    // current state of every system, then this system's slice replaced
    launch_materialize(c->b, c->prec, c->ntiles, c->d_ftmp, c->d_vtmp, c->stream);
    NEFE_CU(cudaStreamSynchronize(c->stream));
    std::vector<double> tmp(3 * (size_t)n);
    for (int which = 0; which < 2; ++which) {
        const double* src = which == 0 ? x : v;
        double* dst = which == 0 ? c->d_ftmp : c->d_vtmp;
        if (!src) continue;
        for (int i = 0; i < n; ++i)
            for (int k = 0; k < 3; ++k) tmp[(size_t)k * n + i] = src[3 * i + k];
        for (int k = 0; k < 3; ++k)
            NEFE_CU(cudaMemcpyAsync(dst + k * N + S.off, tmp.data() + (size_t)k * n, sizeof(double) * n,
                                    cudaMemcpyHostToDevice, c->stream));
        NEFE_CU(cudaStreamSynchronize(c->stream));
    }
    launch_inject(c->b, c->prec, c->ntiles, x ? c->d_ftmp : nullptr, v ? c->d_vtmp : nullptr, c->stream);
    return resetup(c);
}

int nefe_get_trace(nefe_ctx* c, int s, double* buf, long cap, long* n) {
    int rc = check_sys(c, s);
    if (rc) return rc;
    if (!n || (cap > 0 && !buf)) return fail(NEFE_EINVAL, "bad trace buffer");
    if ((rc = setup(c))) return rc;
    if ((rc = set_device(c))) return rc;
    DevState st;
    DevSys S;
    NEFE_CU(cudaMemcpyAsync(&st, c->d_st + s, sizeof(st), cudaMemcpyDeviceToHost, c->stream));
    NEFE_CU(cudaMemcpyAsync(&S, c->d_sys + s, sizeof(S), cudaMemcpyDeviceToHost, c->stream));
    NEFE_CU(cudaStreamSynchronize(c->stream));
    *n = 0;
    if (S.trace_every <= 0 || S.trace_cap <= 0) return NEFE_OK;
    const long long have = std::min<long long>(st.trace_n, S.trace_cap);
    const long long first = st.trace_n - have;
    std::vector<double> ring(9 * (size_t)S.trace_cap);
    NEFE_CU(cudaMemcpy(ring.data(), c->d_trace + 9 * S.trace_off, sizeof(double) * 9 * S.trace_cap,
                       cudaMemcpyDeviceToHost));
    long out = 0;
    for (long long r = first; r < st.trace_n && out < cap; ++r, ++out)
        std::memcpy(buf + 9 * out, ring.data() + 9 * (r % S.trace_cap), sizeof(double) * 9);
    *n = out;
    return NEFE_OK;
}

// Checkpoint file: magic, sizes, then the device arrays in a fixed order.
static const char kMagic[8] = {'N', 'E', 'F', 'E', 'C', 'K', '0', '1'};

struct Blob {
    void* p;
    size_t bytes;
};

static std::vector<Blob> blobs(nefe_ctx* c) {
    const size_t N = c->ntot;
    const size_t v4 = c->prec == NEFE_FP64 ? sizeof(double4) : sizeof(float4);
    const size_t el = c->prec == NEFE_FP64 ? sizeof(double) : sizeof(float);
    std::vector<Blob> all = {{c->d_st, sizeof(DevState) * c->nsys},
            {c->d_acc, sizeof(long long) * c->nsys * ACC_N * kSlots},
            {c->d_pairs, sizeof(DevPair) * std::max<size_t>(1, c->pairs.size())},
            {c->d_x, sizeof(double) * 3 * N},
            {c->d_v, el * 3 * N},
            {c->d_dhi, el * 3 * N},
            {c->d_dlo, el * 3 * N},
            {c->d_F, v4 * N},
            {c->d_xs, v4 * N},
            {c->d_xa, v4 * N},
            {c->d_sd0, v4 * N},
            {c->d_xi, v4 * N},
            {c->d_q, sizeof(int4) * N},
            {c->d_cell_of, sizeof(int) * N},
            {c->d_perm, sizeof(int) * N},
            {c->d_cell_start, sizeof(int) * (size_t)(c->ncells_total + c->nsys)},
            {c->d_nbr, sizeof(int) * N * (size_t)c->cap},
            {c->d_cnt, sizeof(int) * N},
            {c->d_trace, sizeof(double) * 9 * (size_t)std::max<long long>(1, c->trace_total)},
            {c->d_uf_nbr, c->d_uf_nbr ? sizeof(int) * N * (size_t)kUfCap : 0},
            {c->d_uf_cnt, c->d_uf_cnt ? sizeof(int) * N : 0}};
    std::vector<Blob> out;
    for (const Blob& b : all)
        if (b.bytes > 0) out.push_back(b);   // the UF rows exist only in contexts with UF systems
    return out;
}

int nefe_save(nefe_ctx* c, const char* path) {
    NvtxRange nvtx_("nefe_save");
    if (!c || !path) return fail(NEFE_EINVAL, "NULL argument");
    int rc = setup(c);
    if (rc) return rc;
    if ((rc = set_device(c))) return rc;
    NEFE_CU(cudaStreamSynchronize(c->stream));
    FILE* f = std::fopen(path, "wb");
    if (!f) return fail(NEFE_EINVAL, "cannot open %s for writing", path);
    long long hdr[6] = {c->ntot, c->nsys, (long long)c->pairs.size(), c->prec, c->cap, c->ncells_total};
    bool ok = std::fwrite(kMagic, 1, 8, f) == 8 && std::fwrite(hdr, sizeof(hdr), 1, f) == 1;
    std::vector<char> tmp;
    for (const Blob& bl : blobs(c)) {
        if (!ok) break;
        tmp.resize(bl.bytes);
        if (cudaMemcpy(tmp.data(), bl.p, bl.bytes, cudaMemcpyDeviceToHost) != cudaSuccess) { ok = false; break; }
        ok = std::fwrite(tmp.data(), 1, bl.bytes, f) == bl.bytes;
    }
    std::fclose(f);
    return ok ? NEFE_OK : fail(NEFE_ECUDA, "nefe_save: write failed");
}

int nefe_load(nefe_ctx* c, const char* path) {
    NvtxRange nvtx_("nefe_load");
    if (!c || !path) return fail(NEFE_EINVAL, "NULL argument");
    int rc = setup(c);
    if (rc) return rc;
    if ((rc = set_device(c))) return rc;
    NEFE_CU(cudaStreamSynchronize(c->stream));
    FILE* f = std::fopen(path, "rb");
    if (!f) return fail(NEFE_EINVAL, "cannot open %s", path);
    char magic[8];
    long long hdr[6];
    bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, kMagic, 8) == 0 &&
              std::fread(hdr, sizeof(hdr), 1, f) == 1;
    long long want[6] = {c->ntot, c->nsys, (long long)c->pairs.size(), c->prec, c->cap, c->ncells_total};
    if (ok && std::memcmp(hdr, want, sizeof(hdr)) != 0) {
        std::fclose(f);
        return fail(NEFE_EINVAL, "nefe_load: checkpoint does not match this context");
    }
    std::vector<char> tmp;
    for (const Blob& bl : blobs(c)) {
        if (!ok) break;
        tmp.resize(bl.bytes);
        ok = std::fread(tmp.data(), 1, bl.bytes, f) == bl.bytes &&
             cudaMemcpy(bl.p, tmp.data(), bl.bytes, cudaMemcpyHostToDevice) == cudaSuccess;
    }
    std::fclose(f);
    return ok ? NEFE_OK : fail(NEFE_EINVAL, "nefe_load: truncated or unreadable checkpoint");
}

// Step-level refinement of the kernel-level choice: the two fastest pass-A variants with each
// pass-B variant run as real captured steps (2 x kGraphSteps, timed after one warm replay) on
// a device snapshot of the whole dynamic state (the checkpoint blobs), which is restored after
// every candidate, so the context continues bit for bit where it was.  A kernel timed alone
// can rank the variants differently from the same kernel inside the step.  Without memory for
// the snapshot the kernel-level choice stands.
static int refine_in_steps(nefe_ctx* c, const std::vector<std::pair<double, int>>& ranked_a) {
    const std::vector<Blob> bl = blobs(c);
    size_t total = 0;
    for (const Blob& x : bl) total += (x.bytes + 255) / 256 * 256;
    char* snap = nullptr;
    if (cudaMalloc(&snap, total) != cudaSuccess) {
        cudaGetLastError();
        return NEFE_OK;
    }
    auto copy = [&](bool save) {
        size_t off = 0;
        for (const Blob& x : bl) {
            if (save) cudaMemcpyAsync(snap + off, x.p, x.bytes, cudaMemcpyDeviceToDevice, c->stream);
            else cudaMemcpyAsync(x.p, snap + off, x.bytes, cudaMemcpyDeviceToDevice, c->stream);
            off += (x.bytes + 255) / 256 * 256;
        }
    };
    copy(true);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const bool prof = c->profiling;
    c->profiling = false;
    const long launches = c->launches;
    double best = 1e30;
    int best_a = c->lanes, best_b = c->glanes;
    int rc = NEFE_OK;
    for (size_t ka = 0; ka < ranked_a.size() && ka < 2 && rc == NEFE_OK; ++ka) {
        for (int lb : {1, 2, 4, 8}) {
            if (ranked_a[ka].second == 0 && lb != 1) continue;   // the scatter form has one pass B
            c->lanes = ranked_a[ka].second;
            c->glanes = lb;
            drop_graph(c);
            if ((rc = nefe_run(c, kGraphSteps))) break;
            cudaEventRecord(e0, c->stream);
            if ((rc = nefe_run(c, 2 * kGraphSteps))) break;
            cudaEventRecord(e1, c->stream);
            float ms = 1e30f;
            if (cudaEventSynchronize(e1) == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
            const double us = 1000.0 * ms / (2 * kGraphSteps);
            if (us < best) { best = us; best_a = ranked_a[ka].second; best_b = lb; }
            copy(false);
        }
    }
    // The list build keeps its form (one warp per cell, the default: it runs as the single-launch
    // cooperative rebuild): timed over a few real steps its forms rank by noise whenever no list
    // happens to be rebuilt in the window.
    // then the rebuild policy with the chosen lanes (its effect too is seen only in real steps)
    int best_r = c->rebuild_all;
    if (rc == NEFE_OK) {
        const int other = 1 - c->rebuild_all;
        c->lanes = best_a;
        c->glanes = best_b;
        c->b.rebuild_all = other;
        drop_graph(c);
        if ((rc = nefe_run(c, kGraphSteps)) == NEFE_OK) {
            cudaEventRecord(e0, c->stream);
            if ((rc = nefe_run(c, 2 * kGraphSteps)) == NEFE_OK) {
                cudaEventRecord(e1, c->stream);
                float ms = 1e30f;
                if (cudaEventSynchronize(e1) == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
                const double us = 1000.0 * ms / (2 * kGraphSteps);
                if (us < best) { best = us; best_r = other; }
                copy(false);
            }
        }
    }
    c->rebuild_all = best_r;
    c->b.rebuild_all = best_r;
    cudaStreamSynchronize(c->stream);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(snap);
    c->profiling = prof;
    c->launches = launches;
    drop_graph(c);
    if (rc) return rc;
    c->lanes = best_a;
    c->glanes = best_b;
    c->tune_us = best;
    NEFE_CU(cudaGetLastError());
    return NEFE_OK;
}

int nefe_autotune(nefe_ctx* c) {
    NvtxRange nvtx_("nefe_autotune");
    if (!c) return fail(NEFE_EINVAL, "context is NULL");
    int rc = setup(c);
    if (rc) return rc;
    if ((rc = set_device(c))) return rc;
    Bufs b = c->b;
    b.acc = c->d_acc_tmp;
    b.f_out = c->d_ftmp;
    b.e_atom = nullptr;
    cudaEvent_t e0, e1;
    NEFE_CU(cudaEventCreate(&e0));
    NEFE_CU(cudaEventCreate(&e1));
    // best of three trials of five launches each, after two warm-up launches
    auto time_us = [&](auto&& launch) {
        for (int w = 0; w < 2; ++w) launch();
        double best_trial = 1e30;
        for (int trial = 0; trial < 3; ++trial) {
            cudaEventRecord(e0, c->stream);
            const int reps = 5;
            for (int r = 0; r < reps; ++r) launch();
            cudaEventRecord(e1, c->stream);
            float ms = 1e30f;
            if (cudaEventSynchronize(e1) == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
            best_trial = std::min(best_trial, 1000.0 * ms / reps);
        }
        return best_trial;
    };
    const int cand[6] = {0, 1, 4, 8, 16, 32};
    double best = 1e30;
    int best_l = c->lanes;
    std::vector<std::pair<double, int>> ranked_a;   // (time, lanes) of every pass-A variant
    // the scatter form's pass A is timed together with its pass B (k_finish, which clears the
    // accumulators); the gather form's pass B is timed below
    const size_t el_ = c->prec == NEFE_FP64 ? sizeof(double) : sizeof(float);
    void *tv0 = nullptr, *tf0 = nullptr;
    NEFE_CU(cudaMalloc(&tv0, el_ * 3 * c->ntot));
    NEFE_CU(cudaMalloc(&tf0, 4 * el_ * c->ntot));
    NEFE_CU(cudaMemcpyAsync(tv0, c->d_v, el_ * 3 * c->ntot, cudaMemcpyDeviceToDevice, c->stream));
    Bufs b0 = b;
    b0.v = tv0;
    b0.F = tf0;
    double scatter_us = 1e30;
    for (int l : cand) {
        if (c->prec == NEFE_FP64 && (l == 0 || l == 1 || l == 4)) continue;
        double us;
        if (l == 0) {
            us = time_us([&] {
                launch_edges(b0, c->prec, 0, c->ntiles, FM_FORCES, c->stream, &c->launches);
                launch_gather(b0, c->prec, 0, c->ntiles, FM_STEP, c->stream, &c->launches);
            });
            scatter_us = us;
        } else {
            us = time_us([&] { launch_edges(b, c->prec, l, c->ntiles, FM_FORCES, c->stream, &c->launches); });
        }
        ranked_a.push_back({us, l});
        if (us < best) { best = us; best_l = l; }
    }
    NEFE_CU(cudaStreamSynchronize(c->stream));
    cudaFree(tv0);
    cudaFree(tf0);
    std::sort(ranked_a.begin(), ranked_a.end());
    launch_edges(b, c->prec, best_l == 0 ? 1 : best_l, c->ntiles, FM_FORCES, c->stream, &c->launches);
    double best_g = 1e30;
    int best_gl = c->glanes;
    {
        // pass B is timed in its step form (springs, Langevin, kick) on scratch copies of the
        // velocities and the force, so the state is left as it was
        const size_t el = c->prec == NEFE_FP64 ? sizeof(double) : sizeof(float);
        const size_t v4 = 4 * el;
        void *tv = nullptr, *tf = nullptr;
        NEFE_CU(cudaMalloc(&tv, el * 3 * c->ntot));
        NEFE_CU(cudaMalloc(&tf, v4 * c->ntot));
        NEFE_CU(cudaMemcpyAsync(tv, c->d_v, el * 3 * c->ntot, cudaMemcpyDeviceToDevice, c->stream));
        Bufs bs = b;
        bs.v = tv;
        bs.F = tf;
        // each variant right after pass A, as in a step (pass B reads what pass A just wrote);
        // the scatter form was timed with its own pass B above
        const int la = best_l == 0 ? 1 : best_l;
        double base_a = best;
        for (const auto& r : ranked_a)
            if (r.second == la) base_a = r.first;
        for (int l : {1, 2, 4, 8}) {
            const double us = time_us([&] {
                launch_edges(b, c->prec, la, c->ntiles, FM_FORCES, c->stream, &c->launches);
                launch_gather(bs, c->prec, l, c->ntiles, FM_STEP, c->stream, &c->launches);
            });
            if (us < best_g) { best_g = us; best_gl = l; }
        }
        best_g -= base_a;
        // a gather-form pair faster than the scatter form (pass A + its pass B) replaces it
        if (best_l == 0 && base_a + best_g < scatter_us) best_l = la;
        if (best_l == 0) best_g = 0.0;
        NEFE_CU(cudaStreamSynchronize(c->stream));
        cudaFree(tv);
        cudaFree(tf);
    }
    // the list build's lanes are chosen in real steps only (refine_in_steps): a full rebuild,
    // the only thing timeable here, ranks them differently from the partial rebuilds of a run
    const int best_ll = c->llanes;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    NEFE_CU(cudaGetLastError());
    if (best_l != c->lanes || best_gl != c->glanes || best_ll != c->llanes) drop_graph(c);
    c->lanes = best_l;
    c->glanes = best_gl;
    c->llanes = best_ll;
    c->b.list_lanes = best_ll;
    c->tune_us = best + best_g;
    return refine_in_steps(c, ranked_a);
}

int nefe_get_lanes(nefe_ctx* c, int lanes[3]) {
    if (!c || !lanes) return fail(NEFE_EINVAL, "NULL argument");
    lanes[0] = c->lanes;
    lanes[1] = c->glanes;
    lanes[2] = c->llanes;
    return NEFE_OK;
}

int nefe_get_tuning(nefe_ctx* c, int* lanes, double* best_us) {
    if (!c) return fail(NEFE_EINVAL, "context is NULL");
    if (lanes) *lanes = c->lanes;
    if (best_us) *best_us = c->tune_us;
    return NEFE_OK;
}

int nefe_set_tuning(nefe_ctx* c, int lanes) {
    if (!c) return fail(NEFE_EINVAL, "context is NULL");
    if (!lanes_supported(lanes) || (c->prec == NEFE_FP64 && (lanes == 0 || lanes == 1 || lanes == 4)))
        return fail(NEFE_EINVAL, "unsupported lanes per atom %d", lanes);
    if (lanes != c->lanes) drop_graph(c);
    c->lanes = lanes;
    return NEFE_OK;
}

int nefe_set_state_all(nefe_ctx* c, const double* x, const double* v) {
    NvtxRange nvtx_("nefe_set_state_all");
    if (!c) return fail(NEFE_EINVAL, "context is NULL");
    int rc = setup(c);
    if (rc) return rc;
    if ((rc = set_device(c))) return rc;
    const size_t N = c->ntot;
    for (int which = 0; which < 2; ++which) {
        const double* src = which == 0 ? x : v;
        if (!src) continue;
        // host (N,3) -> device staging -> SoA -> state
        NEFE_CU(cudaMemcpyAsync(c->d_shd, src, sizeof(double) * 3 * N, cudaMemcpyHostToDevice, c->stream));
        launch_aos_soa(static_cast<const double*>(c->d_shd), which == 0 ? c->d_ftmp : c->d_vtmp, (int)N, 1, c->stream);
    }
    launch_inject(c->b, c->prec, c->ntiles, x ? c->d_ftmp : nullptr, v ? c->d_vtmp : nullptr, c->stream);
    return resetup(c);
}

int nefe_get_state_all(nefe_ctx* c, double* x, double* v) {
    NvtxRange nvtx_("nefe_get_state_all");
    if (!c) return fail(NEFE_EINVAL, "context is NULL");
    int rc = setup(c);
    if (rc) return rc;
    if ((rc = set_device(c))) return rc;
    const size_t N = c->ntot;
    launch_materialize(c->b, c->prec, c->ntiles, c->d_ftmp, c->d_vtmp, c->stream);
    for (int which = 0; which < 2; ++which) {
        double* dst = which == 0 ? x : v;
        if (!dst) continue;
        double* stage = static_cast<double*>(c->d_shd);
        launch_aos_soa(which == 0 ? c->d_ftmp : c->d_vtmp, stage, (int)N, 0, c->stream);
        NEFE_CU(cudaMemcpyAsync(dst, stage, sizeof(double) * 3 * N, cudaMemcpyDeviceToHost, c->stream));
    }
    NEFE_CU(cudaStreamSynchronize(c->stream));
    return NEFE_OK;
}

int nefe_get_results_all(nefe_ctx* c, nefe_results* out, int count) {
    NvtxRange nvtx_("nefe_get_results_all");
    if (!c || (count > 0 && !out)) return fail(NEFE_EINVAL, "bad argument");
    if (count > (int)c->sys.size()) return fail(NEFE_EINVAL, "count above the number of systems");
    int rc = setup(c);
    if (rc) return rc;
    if ((rc = set_device(c))) return rc;
    launch_group(c->b, c->d_groups, c->ngroups, 2, c->stream, &c->launches);
    std::vector<DevState> st(count > 0 ? count : 1);
    std::vector<DevSys> S(count > 0 ? count : 1);
    if (count > 0) {
        NEFE_CU(cudaMemcpyAsync(st.data(), c->d_st, sizeof(DevState) * count, cudaMemcpyDeviceToHost, c->stream));
        NEFE_CU(cudaMemcpyAsync(S.data(), c->d_sys, sizeof(DevSys) * count, cudaMemcpyDeviceToHost, c->stream));
    }
    NEFE_CU(cudaStreamSynchronize(c->stream));
    for (int s = 0; s < count; ++s) fill_results(S[s], st[s], out + s);
    return NEFE_OK;
}

int nefe_get_shell_stats(nefe_ctx* c, double* mean_count, int* max_count) {
    if (!c) return fail(NEFE_EINVAL, "context is NULL");
    int rc = setup(c);
    if (rc) return rc;
    if ((rc = set_device(c))) return rc;
    std::vector<int> shn(c->ntot);
    std::vector<DevSys> S(c->nsys);
    NEFE_CU(cudaMemcpyAsync(shn.data(), c->d_shn, sizeof(int) * c->ntot, cudaMemcpyDeviceToHost, c->stream));
    NEFE_CU(cudaMemcpyAsync(S.data(), c->d_sys, sizeof(DevSys) * c->nsys, cudaMemcpyDeviceToHost, c->stream));
    NEFE_CU(cudaStreamSynchronize(c->stream));
    double sum = 0.0;
    long long n = 0;
    int mx = 0;
    for (int s = 0; s < c->nsys; ++s) {
        if (S[s].pot != POT_SW) continue;
        for (int i = 0; i < S[s].n; ++i) {
            const int v = shn[S[s].off + i];
            sum += v;
            mx = std::max(mx, v);
        }
        n += S[s].n;
    }
    if (mean_count) *mean_count = n > 0 ? sum / (double)n : 0.0;
    if (max_count) *max_count = mx;
    return NEFE_OK;
}

int nefe_get_list_stats(nefe_ctx* c, int sys, double* mean_count, int* max_count, long* builds) {
    if (!c) return fail(NEFE_EINVAL, "context is NULL");
    if (sys != -1) {
        int rc = check_sys(c, sys);
        if (rc) return rc;
    }
    int rc = setup(c);
    if (rc) return rc;
    if ((rc = set_device(c))) return rc;
    std::vector<int> cnt(c->ntot);
    std::vector<DevState> st(c->nsys);
    std::vector<DevSys> S(c->nsys);
    NEFE_CU(cudaMemcpyAsync(cnt.data(), c->d_cnt, sizeof(int) * c->ntot, cudaMemcpyDeviceToHost, c->stream));
    NEFE_CU(cudaMemcpyAsync(st.data(), c->d_st, sizeof(DevState) * c->nsys, cudaMemcpyDeviceToHost, c->stream));
    NEFE_CU(cudaMemcpyAsync(S.data(), c->d_sys, sizeof(DevSys) * c->nsys, cudaMemcpyDeviceToHost, c->stream));
    NEFE_CU(cudaStreamSynchronize(c->stream));
    double sum = 0.0;
    long long n = 0, nb = 0;
    int mx = 0;
    for (int s = 0; s < c->nsys; ++s) {
        if (sys != -1 && s != sys) continue;
        for (int i = 0; i < S[s].n; ++i) {
            const int v = cnt[S[s].off + i];
            sum += v;
            mx = std::max(mx, v);
        }
        n += S[s].n;
        nb += st[s].nbuild;
    }
    if (mean_count) *mean_count = n > 0 ? sum / (double)n : 0.0;
    if (max_count) *max_count = mx;
    if (builds) *builds = (long)nb;
    return NEFE_OK;
}

int nefe_set_profiling(nefe_ctx* c, int enable) {
    if (!c) return fail(NEFE_EINVAL, "context is NULL");
    int rc = set_device(c);
    if (rc) return rc;
    if ((bool)enable == c->profiling) return NEFE_OK;
    drop_graph(c);
    c->profiling = enable != 0;
    return NEFE_OK;
}

int nefe_get_profile(nefe_ctx* c, double* us, long* samples) {
    if (!c) return fail(NEFE_EINVAL, "context is NULL");
    if (!c->profiling || c->ev0.empty()) return fail(NEFE_ESTATE, "profiling is not enabled or no graph ran yet");
    int rc = set_device(c);
    if (rc) return rc;
    NEFE_CU(cudaStreamSynchronize(c->stream));
    // per step: the sum over chunks of each pass
    const int nch = std::max<int>(1, (int)c->chunk_tile0.size());
    double ta = 0.0, tb = 0.0;
    long n = 0;
    for (int k = 0; k < kGraphSteps; ++k) {
        bool ok = true;
        double sa = 0.0, sb = 0.0;
        for (int q = 0; q < nch && ok; ++q) {
            const int e = k * nch + q;
            if (e >= (int)c->ev0.size()) { ok = false; break; }
            float ma = 0.f, mb = 0.f;
            if (cudaEventElapsedTime(&ma, c->ev0[e], c->ev1[e]) != cudaSuccess ||
                cudaEventElapsedTime(&mb, c->ev1[e], c->ev2[e]) != cudaSuccess) {
                cudaGetLastError();
                ok = false;
                break;
            }
            sa += ma;
            sb += mb;
        }
        if (ok) { ta += sa; tb += sb; ++n; }
    }
    if (us) {
        us[0] = n > 0 ? 1000.0 * ta / n : 0.0;
        us[1] = n > 0 ? 1000.0 * tb / n : 0.0;
    }
    if (samples) *samples = n;
    return NEFE_OK;
}

int nefe_set_gather_tuning(nefe_ctx* c, int lanes) {
    if (!c) return fail(NEFE_EINVAL, "context is NULL");
    if (lanes != 1 && lanes != 2 && lanes != 4 && lanes != 8)
        return fail(NEFE_EINVAL, "pass B supports 1, 2, 4 or 8 lanes per atom");
    if (lanes != c->glanes) drop_graph(c);
    c->glanes = lanes;
    return NEFE_OK;
}

int nefe_set_rebuild_policy(nefe_ctx* c, int all) {
    if (!c) return fail(NEFE_EINVAL, "context is NULL");
    if (all != 0 && all != 1) return fail(NEFE_EINVAL, "rebuild policy must be 0 or 1");
    if (c->b.rebuild_all != all) drop_graph(c);   // the policy is captured in the step graph
    c->rebuild_all = all;
    c->b.rebuild_all = all;
    return NEFE_OK;
}

int nefe_set_cooperative_rebuild(nefe_ctx* c, int on) {
    if (!c) return fail(NEFE_EINVAL, "context is NULL");
    if (on != 0 && on != 1) return fail(NEFE_EINVAL, "on must be 0 or 1");
    if (c->coop != (on != 0)) drop_graph(c);     // the form is captured in the step graph
    c->coop = on != 0;
    return NEFE_OK;
}

int nefe_get_rebuild_policy(nefe_ctx* c, int* all) {
    if (!c || !all) return fail(NEFE_EINVAL, "NULL argument");
    *all = c->rebuild_all;
    return NEFE_OK;
}

int nefe_set_list_tuning(nefe_ctx* c, int lanes) {
    if (!c) return fail(NEFE_EINVAL, "context is NULL");
    if (lanes != 0 && lanes != 8 && lanes != 16 && lanes != 32)
        return fail(NEFE_EINVAL, "the list build takes 0 (one warp per cell) or 8, 16, 32 lanes per atom");
    if (lanes != c->llanes) drop_graph(c);
    c->llanes = lanes;
    c->b.list_lanes = lanes;
    return NEFE_OK;
}

int nefe_launch_count(nefe_ctx* c, long* count) {
    if (!c || !count) return fail(NEFE_EINVAL, "NULL argument");
    *count = c->launches;
    return NEFE_OK;
}

}  // extern "C"
