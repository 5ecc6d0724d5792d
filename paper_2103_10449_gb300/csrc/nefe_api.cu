// Stateless C-ABI entry points of libnefe (caller-owned device buffers) and error reporting.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "nefe.h"
#include "nefe_dev.h"
#include "nefe_host.h"
#include "nefe_launch.h"
#include "nefe_nvtx.h"

namespace nefe {

static thread_local char g_msg[512] = "no error";

int fail(int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
    va_end(ap);
    return code;
}

int cuda_fail(cudaError_t e, const char* where) {
    if (e == cudaSuccess) return NEFE_OK;
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(NEFE_ENOMEM, "%s: %s", where, cudaGetErrorString(e));
    }
    return fail(NEFE_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

bool valid_params(const nefe_sw_params* p) {
    return p && p->sigma > 0.0 && p->a > 0.0 && p->eps > 0.0 && std::isfinite(p->A) &&
           std::isfinite(p->B) && std::isfinite(p->p) && std::isfinite(p->q) &&
           std::isfinite(p->lambda3) && std::isfinite(p->gamma) && std::isfinite(p->cos0);
}

int check_box(const double box[3], double rcs) {
    for (int k = 0; k < 3; ++k)
        if (!(box[k] > 0.0) || !std::isfinite(box[k]))
            return fail(NEFE_EINVAL, "box length %d is not positive and finite", k);
    if (!(rcs > 0.0)) return fail(NEFE_EINVAL, "rcs must be positive");
    for (int k = 0; k < 3; ++k)
        if (box[k] < 2.0 * rcs)
            return fail(NEFE_EINVAL, "box length %g below 2*rcs = %g", box[k], 2.0 * rcs);
    return NEFE_OK;
}

int prepare1(Scratch1& S, int n, const double box[3], double rcs, int ncell_cap, int prec,
                    bool cells, const nefe_uf_params* uf, double skin) {
    const int ntiles = (n + kTile - 1) / kTile;
    DevSys hs;
    std::memset(&hs, 0, sizeof(hs));
    hs.off = 0; hs.n = n; hs.tile0 = 0; hs.ntile = ntiles; hs.cell0 = 0; hs.ncell_cap = ncell_cap;
    hs.rcs = rcs; hs.pair = -1; hs.prm = 0; hs.mass_e = 1.0;
    hs.rcs2_lo_f = (float)(rcs * rcs) * (1.0f - 1e-4f);
    hs.rcs2_hi_f = (float)(rcs * rcs) * (1.0f + 1e-4f);
    if (uf) {
        fill_uf(hs, *uf, skin, UF_INT);
        hs.pot = POT_UF;
    }
    DevState st;
    std::memset(&st, 0, sizeof(st));
    for (int k = 0; k < 3; ++k) st.box[k] = box[k];
    st.rebuild = 1;
    st.scale_int = 1.0;
    NEFE_CU(S.alloc(&S.sys, sizeof(DevSys)));
    NEFE_CU(S.alloc(&S.st, sizeof(DevState)));
    NEFE_CU(S.alloc(&S.tile_sys, sizeof(int) * (size_t)(ntiles > 0 ? ntiles : 1)));
    NEFE_CU(S.alloc(&S.acc, sizeof(long long) * ACC_N * kSlots));
    NEFE_CU(cudaMemcpyAsync(S.sys, &hs, sizeof(hs), cudaMemcpyHostToDevice, S.s));
    NEFE_CU(cudaMemcpyAsync(S.st, &st, sizeof(st), cudaMemcpyHostToDevice, S.s));
    NEFE_CU(cudaMemsetAsync(S.tile_sys, 0, sizeof(int) * (size_t)(ntiles > 0 ? ntiles : 1), S.s));
    NEFE_CU(cudaMemsetAsync(S.acc, 0, sizeof(long long) * ACC_N * kSlots, S.s));
    const size_t v4 = prec == NEFE_FP64 ? sizeof(double4) : sizeof(float4);
    NEFE_CU(S.alloc(&S.xs, v4 * (size_t)n));
    if (cells) {
        NEFE_CU(S.alloc(&S.xa, v4 * (size_t)n));
        NEFE_CU(S.alloc(&S.xcs, v4 * (size_t)n));
        NEFE_CU(S.alloc(&S.q, sizeof(int4) * (size_t)n));
        NEFE_CU(S.alloc(&S.cell_of, sizeof(int) * (size_t)n));
        NEFE_CU(S.alloc(&S.perm, sizeof(int) * (size_t)n));
        NEFE_CU(S.alloc(&S.cell_start, sizeof(int) * (size_t)(ncell_cap + 1)));
        NEFE_CU(S.alloc(&S.cell_count, sizeof(int) * (size_t)ncell_cap));
        NEFE_CU(S.alloc(&S.cell_cursor, sizeof(int) * (size_t)ncell_cap));
        NEFE_CU(cudaMemsetAsync(S.cell_count, 0, sizeof(int) * (size_t)ncell_cap, S.s));
    }
    return NEFE_OK;
}

Bufs bufs_of(const Scratch1& S, const double* x, int n) {
    Bufs b;
    std::memset(&b, 0, sizeof(b));
    b.sys = S.sys; b.st = S.st; b.acc = S.acc; b.tile_sys = S.tile_sys;
    b.x = const_cast<double*>(x);
    b.xs = S.xs; b.xa = S.xa; b.xcs = S.xcs; b.q = S.q; b.cell_of = S.cell_of; b.perm = S.perm;
    b.shd = S.shd; b.shj = S.shj; b.shn = S.shn; b.P = S.P;
    b.cell_start = S.cell_start; b.cell_count = S.cell_count; b.cell_cursor = S.cell_cursor;
    b.ntot = n; b.swc = S.swc;
    return b;
}

}  // namespace nefe

using namespace nefe;

extern "C" {

const char* nefe_last_error(void) { return g_msg; }

int nefe_sw_params_silicon(nefe_sw_params* out) {
    if (!out) return fail(NEFE_EINVAL, "out is NULL");
    out->eps = 2.1683; out->sigma = 2.0951; out->A = 7.049556277; out->B = 0.6022245584;
    out->p = 4.0; out->q = 0.0; out->a = 1.80; out->lambda3 = 21.0; out->gamma = 1.20;
    out->cos0 = -1.0 / 3.0;
    return NEFE_OK;
}

int nefe_cell_bin(const double* x, int n, const double box[3], double rcs, int ncell3[3],
                  int* cell_of, int* cell_start, int* perm, int ncell_cap, void* stream) {
    NvtxRange nvtx_("nefe_cell_bin");
    if (n < 0 || !box || !ncell3 || (n > 0 && (!x || !cell_of || !perm)) || !cell_start)
        return fail(NEFE_EINVAL, "nefe_cell_bin: bad argument");
    if (n >= (1 << kCodeShift)) return fail(NEFE_EINVAL, "nefe_cell_bin: n above 2^27");
    int rc = check_box(box, rcs);
    if (rc) return rc;
    int n3[3];
    if (!host_grid(box, rcs, n3)) return fail(NEFE_EINVAL, "nefe_cell_bin: fewer than 2 cells on an axis");
    const long long total = (long long)n3[0] * n3[1] * n3[2];
    if (total > ncell_cap) return fail(NEFE_EINVAL, "nefe_cell_bin: %lld cells above capacity %d", total, ncell_cap);
    for (int k = 0; k < 3; ++k) ncell3[k] = n3[k];
    Scratch1 S;
    S.s = (cudaStream_t)stream;
    rc = prepare1(S, n, box, rcs, (int)total, NEFE_FP32, true);
    if (rc) return rc;
    if (n == 0) {
        NEFE_CU(cudaMemsetAsync(cell_start, 0, sizeof(int) * (size_t)(total + 1), S.s));
        return NEFE_OK;
    }
    Bufs b = bufs_of(S, x, n);
    b.cell_of = cell_of; b.perm = perm; b.cell_start = cell_start;
    launch_cells(b, NEFE_FP32, (n + kTile - 1) / kTile, 1, 1, S.s, nullptr);
    NEFE_CU(cudaGetLastError());
    return NEFE_OK;
}

int nefe_neighbor_build(const double* x, int n, const double box[3], double rcs, int cap,
                        int* nbr, int* cnt, int* overflow, void* stream) {
    NvtxRange nvtx_("nefe_neighbor_build");
    if (n < 0 || !box || cap < 1 || cap > kMaxCap || (n > 0 && (!x || !nbr || !cnt)))
        return fail(NEFE_EINVAL, "nefe_neighbor_build: bad argument");
    if (n >= (1 << kCodeShift)) return fail(NEFE_EINVAL, "nefe_neighbor_build: n above 2^27");
    int rc = check_box(box, rcs);
    if (rc) return rc;
    if (overflow) *overflow = 0;
    if (n == 0) return NEFE_OK;
    int n3[3];
    if (!host_grid(box, rcs, n3)) return fail(NEFE_EINVAL, "nefe_neighbor_build: fewer than 2 cells on an axis");
    const long long total = (long long)n3[0] * n3[1] * n3[2];
    if (total > (1LL << 30)) return fail(NEFE_EINVAL, "nefe_neighbor_build: cell grid too large");
    Scratch1 S;
    S.s = (cudaStream_t)stream;
    rc = prepare1(S, n, box, rcs, (int)total, NEFE_FP32, true);
    if (rc) return rc;
    Bufs b = bufs_of(S, x, n);
    b.nbr = nbr; b.cnt = cnt; b.cap = cap;
    launch_cells_and_list(b, NEFE_FP32, (n + kTile - 1) / kTile, 1, 1, S.s, nullptr);
    NEFE_CU(cudaGetLastError());
    DevState st;
    NEFE_CU(cudaMemcpyAsync(&st, S.st, sizeof(st), cudaMemcpyDeviceToHost, S.s));
    NEFE_CU(cudaStreamSynchronize(S.s));
    const int ovf = (st.err & NEFE_ERR_NBR_OVERFLOW) ? 1 : 0;
    if (overflow) *overflow = ovf;
    if (ovf) return fail(NEFE_EOVERFLOW, "nefe_neighbor_build: a row exceeded cap %d", cap);
    return NEFE_OK;
}

int nefe_sw_forces(const double* x, int n, const double box[3], double rcs, const int* nbr,
                   const int* cnt, int cap, const nefe_sw_params* prm, int precision, double* f,
                   double* e_atom, double* energy_virial, int* shell_overflow, void* stream) {
    NvtxRange nvtx_("nefe_sw_forces");
    if (n < 0 || !box || cap < 1 || cap > kMaxCap || !valid_params(prm) ||
        (precision != NEFE_FP32 && precision != NEFE_FP64) || (n > 0 && (!x || !nbr || !cnt || !f)))
        return fail(NEFE_EINVAL, "nefe_sw_forces: bad argument");
    if (prm->a * prm->sigma > rcs) return fail(NEFE_EINVAL, "nefe_sw_forces: a*sigma above rcs");
    int rc = check_box(box, rcs);
    if (rc) return rc;
    if (shell_overflow) *shell_overflow = 0;
    int n3[3];
    if (!host_grid(box, rcs, n3)) return fail(NEFE_EINVAL, "nefe_sw_forces: fewer than 2 cells on an axis");
    const long long total = (long long)n3[0] * n3[1] * n3[2];
    Scratch1 S;
    S.s = (cudaStream_t)stream;
    rc = prepare1(S, n, box, rcs, (int)(total > (1LL << 30) ? (1LL << 30) : total), precision, false);
    if (rc) return rc;
    if (precision == NEFE_FP64) {
        SWc<double> c = make_swc<double>(*prm);
        NEFE_CU(S.alloc(&S.swc, sizeof(c)));
        NEFE_CU(cudaMemcpyAsync(S.swc, &c, sizeof(c), cudaMemcpyHostToDevice, S.s));
    } else {
        SWc<float> c = make_swc<float>(*prm);
        NEFE_CU(S.alloc(&S.swc, sizeof(c)));
        NEFE_CU(cudaMemcpyAsync(S.swc, &c, sizeof(c), cudaMemcpyHostToDevice, S.s));
    }
    if (n > 0) {
        const size_t v4 = precision == NEFE_FP64 ? sizeof(double4) : sizeof(float4);
        NEFE_CU(S.alloc(&S.shd, v4 * (size_t)n * kShell));
        NEFE_CU(S.alloc(&S.shj, sizeof(int) * (size_t)n * kShell));
        NEFE_CU(S.alloc(&S.shn, sizeof(int) * (size_t)n));
        NEFE_CU(S.alloc(&S.P, 3 * v4 * (size_t)n));
        Bufs b = bufs_of(S, x, n);
        b.nbr = const_cast<int*>(nbr); b.cnt = const_cast<int*>(cnt); b.cap = cap;
        b.f_out = f; b.e_atom = e_atom;
        const int ntiles = (n + kTile - 1) / kTile;
        launch_mirror(b, precision, ntiles, S.s, nullptr);
        launch_edges(b, precision, 8, ntiles, FM_FORCES, S.s, nullptr);
        launch_gather(b, precision, 4, ntiles, FM_FORCES, S.s, nullptr);
        NEFE_CU(cudaGetLastError());
    }
    if (energy_virial) launch_decode_ev(S.acc, energy_virial, S.s);
    NEFE_CU(cudaGetLastError());
    if (shell_overflow) {
        DevState st;
        NEFE_CU(cudaMemcpyAsync(&st, S.st, sizeof(st), cudaMemcpyDeviceToHost, S.s));
        NEFE_CU(cudaStreamSynchronize(S.s));
        *shell_overflow = (st.err & NEFE_ERR_SHELL_OVERFLOW) ? 1 : 0;
        if (*shell_overflow) return fail(NEFE_EOVERFLOW, "nefe_sw_forces: shell above 32 neighbours");
    }
    return NEFE_OK;
}

int nefe_sw_energy_grad(const double* x, int n, const double box[3], double rcs, const int* nbr,
                        const int* cnt, int cap, const nefe_sw_params* prm, int precision, double* f,
                        double* energy_grad, void* stream) {
    NvtxRange nvtx_("nefe_sw_energy_grad");
    if (n < 0 || !box || cap < 1 || cap > kMaxCap || !valid_params(prm) || !energy_grad ||
        (precision != NEFE_FP32 && precision != NEFE_FP64) || (n > 0 && (!x || !nbr || !cnt)))
        return fail(NEFE_EINVAL, "nefe_sw_energy_grad: bad argument");
    if (prm->a * prm->sigma > rcs) return fail(NEFE_EINVAL, "nefe_sw_energy_grad: a*sigma above rcs");
    int rc = check_box(box, rcs);
    if (rc) return rc;
    int n3[3];
    if (!host_grid(box, rcs, n3)) return fail(NEFE_EINVAL, "nefe_sw_energy_grad: fewer than 2 cells on an axis");
    const long long total = (long long)n3[0] * n3[1] * n3[2];
    Scratch1 S;
    S.s = (cudaStream_t)stream;
    rc = prepare1(S, n, box, rcs, (int)(total > (1LL << 30) ? (1LL << 30) : total), precision, false);
    if (rc) return rc;
    if (precision == NEFE_FP64) {
        SWc<double> c = make_swc<double>(*prm);
        NEFE_CU(S.alloc(&S.swc, sizeof(c)));
        NEFE_CU(cudaMemcpyAsync(S.swc, &c, sizeof(c), cudaMemcpyHostToDevice, S.s));
    } else {
        SWc<float> c = make_swc<float>(*prm);
        NEFE_CU(S.alloc(&S.swc, sizeof(c)));
        NEFE_CU(cudaMemcpyAsync(S.swc, &c, sizeof(c), cudaMemcpyHostToDevice, S.s));
    }
    if (n > 0) {
        const size_t v4 = precision == NEFE_FP64 ? sizeof(double4) : sizeof(float4);
        double* fo = f;
        if (!fo) NEFE_CU(S.alloc(&fo, sizeof(double) * 3 * (size_t)n));
        NEFE_CU(S.alloc(&S.shd, v4 * (size_t)n * kShell));
        NEFE_CU(S.alloc(&S.shj, sizeof(int) * (size_t)n * kShell));
        NEFE_CU(S.alloc(&S.shn, sizeof(int) * (size_t)n));
        NEFE_CU(S.alloc(&S.P, 3 * v4 * (size_t)n));
        Bufs b = bufs_of(S, x, n);
        b.nbr = const_cast<int*>(nbr); b.cnt = const_cast<int*>(cnt); b.cap = cap;
        b.f_out = fo; b.e_atom = nullptr; b.want_grad = 1;
        const int ntiles = (n + kTile - 1) / kTile;
        launch_mirror(b, precision, ntiles, S.s, nullptr);
        launch_edges(b, precision, 8, ntiles, FM_FORCES, S.s, nullptr);
        launch_gather(b, precision, 4, ntiles, FM_FORCES, S.s, nullptr);
        NEFE_CU(cudaGetLastError());
    }
    launch_decode_grad(S.acc, energy_grad, S.s);
    NEFE_CU(cudaGetLastError());
    DevState st;
    NEFE_CU(cudaMemcpyAsync(&st, S.st, sizeof(st), cudaMemcpyDeviceToHost, S.s));
    NEFE_CU(cudaStreamSynchronize(S.s));
    if (st.err & NEFE_ERR_SHELL_OVERFLOW)
        return fail(NEFE_EOVERFLOW, "nefe_sw_energy_grad: shell above 32 neighbours");
    if (st.err & NEFE_ERR_NAN) return fail(NEFE_ENAN, "nefe_sw_energy_grad: non-finite sum");
    return NEFE_OK;
}

int nefe_uf_forces(const double* x, int n, const double box[3], double rcs, double skin,
                   const nefe_uf_params* uf, int precision, double* f, double* e_atom,
                   double* energy_virial, void* stream) {
    NvtxRange nvtx_("nefe_uf_forces");
    if (n < 0 || !box || !valid_uf(uf) || !(skin >= 0.0) || (precision != NEFE_FP32 && precision != NEFE_FP64) ||
        (n > 0 && (!x || !f)))
        return fail(NEFE_EINVAL, "nefe_uf_forces: bad argument");
    if (n >= (1 << kUfShift)) return fail(NEFE_EINVAL, "nefe_uf_forces: n above 2^25");
    int rc = check_box(box, rcs);
    if (rc) return rc;
    const double R = uf->rc + skin;
    if (R > 2.0 * rcs) return fail(NEFE_EINVAL, "nefe_uf_forces: rc + skin = %g above 2 rcs = %g", R, 2.0 * rcs);
    int n3[3];
    if (!host_grid(box, rcs, n3)) return fail(NEFE_EINVAL, "nefe_uf_forces: fewer than 2 cells on an axis");
    for (int k = 0; k < 3; ++k) {
        if (n3[k] < 5) return fail(NEFE_EINVAL, "nefe_uf_forces: fewer than 5 cells on an axis");
        if (box[k] < 2.0 * R) return fail(NEFE_EINVAL, "nefe_uf_forces: box below 2 (rc + skin)");
    }
    const long long total = (long long)n3[0] * n3[1] * n3[2];
    if (total > (1LL << 30)) return fail(NEFE_EINVAL, "nefe_uf_forces: cell grid too large");
    Scratch1 S;
    S.s = (cudaStream_t)stream;
    rc = prepare1(S, n, box, rcs, (int)total, precision, true, uf, skin);
    if (rc) return rc;
    if (n > 0) {
        int* uf_nbr = nullptr;
        int* uf_cnt = nullptr;
        NEFE_CU(S.alloc(&uf_nbr, sizeof(int) * (size_t)n * kUfCap));
        NEFE_CU(S.alloc(&uf_cnt, sizeof(int) * (size_t)n));
        Bufs b = bufs_of(S, x, n);
        b.uf_nbr = uf_nbr; b.uf_cnt = uf_cnt; b.uf_tiles = nullptr;
        b.f_out = f; b.e_atom = e_atom;
        const int ntiles = (n + kTile - 1) / kTile;
        launch_cells(b, precision, ntiles, 1, 1, S.s, nullptr);
        launch_uf_list(b, precision, ntiles, S.s, nullptr);
        launch_uf(b, precision, ntiles, FM_FORCES, S.s, nullptr);
        NEFE_CU(cudaGetLastError());
    }
    if (energy_virial) launch_decode_ev(S.acc, energy_virial, S.s);
    NEFE_CU(cudaGetLastError());
    DevState st;
    NEFE_CU(cudaMemcpyAsync(&st, S.st, sizeof(st), cudaMemcpyDeviceToHost, S.s));
    NEFE_CU(cudaStreamSynchronize(S.s));
    if (st.err & NEFE_ERR_NBR_OVERFLOW) return fail(NEFE_EOVERFLOW, "nefe_uf_forces: a row exceeded %d", kUfCap);
    if (st.err & (NEFE_ERR_BOX | NEFE_ERR_CELL)) return fail(NEFE_EINVAL, "nefe_uf_forces: cell grid error");
    return NEFE_OK;
}

int nefe_check_barrier_timeout(int device, double limit_ms) {
    if (!(limit_ms > 0.0 && limit_ms <= 1000.0)) return fail(NEFE_EINVAL, "limit_ms must be in (0, 1000]");
    NEFE_CU(cudaSetDevice(device));
    const int r = check_barrier_timeout(limit_ms);
    if (r < 0) return fail(NEFE_ECUDA, "barrier check: CUDA error");
    return r ? fail(NEFE_ETIMEOUT, "the barrier gave up by its limit (expected)") : NEFE_OK;
}

int nefe_langevin_noise(uint64_t seed, uint64_t sys_id, uint64_t step, int n, int precision,
                        double* xi, void* stream) {
    NvtxRange nvtx_("nefe_langevin_noise");
    if (n < 0 || (n > 0 && !xi) || (precision != NEFE_FP32 && precision != NEFE_FP64))
        return fail(NEFE_EINVAL, "nefe_langevin_noise: bad argument");
    launch_noise(seed, sys_id, step, n, precision, xi, (cudaStream_t)stream);
    NEFE_CU(cudaGetLastError());
    return NEFE_OK;
}

}  // extern "C"
