// Host helpers shared by the C-ABI translation units of libnefe.
#pragma once
#include <cuda_runtime.h>
#include <cmath>
#include <vector>

#include "nefe.h"
#include "nefe_dev.h"
#include "nefe_launch.h"

namespace nefe {

// Records a message for nefe_last_error() and returns code.
int fail(int code, const char* fmt, ...);
// Maps a CUDA error to NEFE_ECUDA with a message (NEFE_OK when e == cudaSuccess).
int cuda_fail(cudaError_t e, const char* where);

#define NEFE_CU(call)                                   \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

// Cell grid of the list-build rule (same arithmetic as the device): floor(L/rcs), reduced
// while L/n < rcs (1 + 1e-9).  Returns false when an axis gets fewer than 2 cells.
inline bool host_grid(const double box[3], double rcs, int n3[3]) {
    bool ok = true;
    for (int k = 0; k < 3; ++k) {
        // clamped before the conversion to int (a huge box would overflow it); so many cells
        // exceed every capacity and are rejected by the callers' cell-count check
        const double q = std::floor(box[k] / rcs);
        int m = q < (double)(1 << 20) ? (int)q : (1 << 20);
        while (m > 0 && box[k] / (double)m < rcs * (1.0 + 1e-9)) --m;
        if (m < 2) ok = false;
        n3[k] = m < 2 ? 2 : m;
    }
    return ok;
}

template <typename T>
inline SWc<T> make_swc(const nefe_sw_params& p) {
    SWc<T> c;
    c.inv_sig = (T)(1.0 / p.sigma);
    c.a = (T)p.a;
    const double rc = p.a * p.sigma;
    c.rc2 = (T)(rc * rc);
    c.epsA = (T)(p.eps * p.A);
    c.B = (T)p.B;
    c.p = (T)p.p;
    c.q = (T)p.q;
    c.epslam = (T)(p.eps * p.lambda3);
    c.gam = (T)p.gamma;
    c.c0 = (T)p.cos0;
    c.eps = (T)p.eps;
    c.A = (T)p.A;
    c.lam3 = (T)p.lambda3;
    // FP32 path: an edge whose three-body factor exp(gamma/(s - a)) is below 1e-12 adds forces
    // of order 1e-8 eV/A (pair and triplet), far below FP32 resolution, so it is dropped:
    // s_act = a + gamma / ln(1e-12).  FP64 path: only the last 1e-12 sigma before the cutoff
    // (where the terms underflow to 0) is dropped.
    if (sizeof(T) == 4) c.s_act = (T)(p.a + p.gamma / std::log(1e-12));
    else c.s_act = (T)(p.a - 1e-12);
    const double ract = (double)c.s_act * p.sigma;
    c.act2 = (T)(ract * ract < rc * rc ? ract * ract : rc * rc);
    c.int_pq = (p.p == 4.0 && p.q == 0.0) ? 1 : 0;
    return c;
}

bool valid_params(const nefe_sw_params* p);

// Uhlenbeck-Ford constants of a system (mode UF_INT or UF_REF; list radius rc + skin).
inline void fill_uf(DevSys& d, const nefe_uf_params& uf, double skin, int mode) {
    const double kT = kB * uf.T;
    const double R = uf.rc + skin;
    d.uf_mode = mode;
    d.uf_pk = uf.p * kT;
    d.uf_is2 = 1.0 / (uf.sigma * uf.sigma);
    d.uf_rc2 = uf.rc * uf.rc;
    d.uf_shift = -d.uf_pk * std::log(-std::expm1(-d.uf_rc2 * d.uf_is2));
    d.uf_R2 = R * R;
    d.uf_pk_f = (float)d.uf_pk;
    d.uf_is2_f = (float)d.uf_is2;
    d.uf_rc2_f = (float)d.uf_rc2;
    d.uf_shift_f = (float)d.uf_shift;
    d.uf_R2_f = (float)d.uf_R2;
}
inline bool valid_uf(const nefe_uf_params* u) {
    return u && u->p > 0.0 && u->sigma > 0.0 && u->T > 0.0 && u->rc > 0.0 && std::isfinite(u->p) &&
           std::isfinite(u->sigma) && std::isfinite(u->T) && std::isfinite(u->rc);
}

// Single-system descriptors and scratch for the stateless calls and the adjoint context
// (stream-ordered allocations, released on the same stream).
struct Scratch1 {
    DevSys* sys = nullptr;
    DevState* st = nullptr;
    int* tile_sys = nullptr;
    long long* acc = nullptr;
    void* swc = nullptr;
    int4* q = nullptr;
    void* xs = nullptr;
    void* xa = nullptr;
    void* xcs = nullptr;
    void* shd = nullptr;
    int* shj = nullptr;
    int* shn = nullptr;
    void* P = nullptr;
    int* cell_of = nullptr;
    int* perm = nullptr;
    int* cell_start = nullptr;
    int* cell_count = nullptr;
    int* cell_cursor = nullptr;
    cudaStream_t s = nullptr;
    std::vector<void*> owned;

    template <typename P>
    cudaError_t alloc(P** p, size_t bytes) {
        void* q = nullptr;
        cudaError_t e = cudaMallocAsync(&q, bytes < 16 ? 16 : bytes, s);
        if (e == cudaSuccess) owned.push_back(q);
        *p = static_cast<P*>(q);
        return e;
    }
    ~Scratch1() {
        for (void* p : owned) cudaFreeAsync(p, s);
    }
};

// NEFE_OK when every box length is positive, finite and at least 2 rcs.
int check_box(const double box[3], double rcs);
// Sets up the one-system descriptors, the tile table and (cells) the cell arrays.
// With uf, the system carries a Uhlenbeck-Ford term as U_int (list radius uf->rc + skin).
int prepare1(Scratch1& S, int n, const double box[3], double rcs, int ncell_cap, int prec, bool cells,
             const nefe_uf_params* uf = nullptr, double skin = 0.0);
// Launch arguments over S for n atoms at FP64 positions x.
Bufs bufs_of(const Scratch1& S, const double* x, int n);

}  // namespace nefe
