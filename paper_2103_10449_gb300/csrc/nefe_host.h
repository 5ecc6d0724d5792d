// Host helpers shared by the C-ABI translation units of libnefe.
#pragma once
#include <cuda_runtime.h>
#include <cmath>

#include "nefe.h"
#include "nefe_dev.h"

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
        int m = (int)std::floor(box[k] / rcs);
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

}  // namespace nefe
