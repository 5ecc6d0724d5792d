// Differentiation of the switching work W(theta) = sum_k dH/dlambda(x_k) (lambda_{k+1} - lambda_k)
// (Eq. Wdyn, left point) with respect to the SW parameters theta = (A, B, p, q, a, lambda3,
// gamma), through the Langevin velocity-Verlet trajectory with the thermostat noise held fixed.
//
// Building block: one FP64 kernel evaluates the SW energy, forces and dU/dtheta in dual numbers
// v + eps d, the dual direction being a displacement w of every atom together with a parameter
// direction dtheta.  The dual parts are then
//   F'  = J w + (dF/dtheta) dtheta          (J = dF/dx = -Hessian, symmetric)
//   E'  = -F . w + (dU/dtheta) . dtheta
//   G'  = (d2U/dtheta dx) w + (d2U/dtheta2) dtheta    (G = dU/dtheta)
// which are the Hessian-vector and mixed products that both the tangent-linear run and the
// reverse (adjoint) sweep need.  The kernel is gather-only (atom i sums the pair terms, the
// triplets centred on it and the triplets centred on each neighbour in which it is a leg), so
// every output is reproducible bit for bit.
//
// The adjoint context integrates its own FP64 NVT trajectory (Frenkel-Ladd or reversible
// scaling, same update as the engine's FP64 path), keeps (x, v, F) every K_c steps, and in the
// reverse sweep recomputes each segment from its checkpoint before stepping the adjoint
// variables back through it.
#include <cstddef>
#include <cstdint>
#include <cstring>
#include <vector>

#include "nefe.h"
#include "nefe_dev.h"
#include "nefe_host.h"
#include "nefe_launch.h"
#include "nefe_nvtx.h"

namespace nefe {
namespace ad {

constexpr int kAdThreads = 128;
constexpr int kAdShell = 32;
constexpr int kRed = 16;     // [E, E', G(7), G'(7)]

// ---------------------------------------------------------------------------- dual numbers
struct Dd {
    double v, d;
};
__host__ __device__ __forceinline__ Dd mk(double v, double d) { Dd r; r.v = v; r.d = d; return r; }
__device__ __forceinline__ Dd operator+(Dd a, Dd b) { return mk(a.v + b.v, a.d + b.d); }
__device__ __forceinline__ Dd operator-(Dd a, Dd b) { return mk(a.v - b.v, a.d - b.d); }
__device__ __forceinline__ Dd operator-(Dd a) { return mk(-a.v, -a.d); }
__device__ __forceinline__ Dd operator*(Dd a, Dd b) { return mk(a.v * b.v, a.v * b.d + a.d * b.v); }
__device__ __forceinline__ Dd operator*(double s, Dd a) { return mk(s * a.v, s * a.d); }
__device__ __forceinline__ Dd operator*(Dd a, double s) { return mk(s * a.v, s * a.d); }
__device__ __forceinline__ Dd operator+(Dd a, double s) { return mk(a.v + s, a.d); }
__device__ __forceinline__ Dd operator-(Dd a, double s) { return mk(a.v - s, a.d); }
__device__ __forceinline__ Dd& operator+=(Dd& a, Dd b) { a.v += b.v; a.d += b.d; return a; }
__device__ __forceinline__ Dd& operator-=(Dd& a, Dd b) { a.v -= b.v; a.d -= b.d; return a; }

__device__ __forceinline__ double val(double a) { return a; }
__device__ __forceinline__ double val(Dd a) { return a.v; }
__device__ __forceinline__ double dua(double) { return 0.0; }
__device__ __forceinline__ double dua(Dd a) { return a.d; }
template <typename T> __device__ __forceinline__ T lift(double v, double d);
template <> __device__ __forceinline__ double lift<double>(double v, double) { return v; }
template <> __device__ __forceinline__ Dd lift<Dd>(double v, double d) { return mk(v, d); }

__device__ __forceinline__ double f_exp(double a) { return exp(a); }
__device__ __forceinline__ Dd f_exp(Dd a) { const double e = exp(a.v); return mk(e, e * a.d); }
__device__ __forceinline__ double f_log(double a) { return log(a); }
__device__ __forceinline__ Dd f_log(Dd a) { return mk(log(a.v), a.d / a.v); }
__device__ __forceinline__ double f_sqrt(double a) { return sqrt(a); }
__device__ __forceinline__ Dd f_sqrt(Dd a) { const double s = sqrt(a.v); return mk(s, a.d / (2.0 * s)); }
__device__ __forceinline__ double f_rcp(double a) { return 1.0 / a; }
__device__ __forceinline__ Dd f_rcp(Dd a) { const double r = 1.0 / a.v; return mk(r, -a.d * r * r); }

// SW parameters; the seven differentiable ones carry the parameter direction as dual part.
template <typename T>
struct SWad {
    double eps, inv_sig, c0, rc2;
    T A, B, p, q, a, lam, gam;
};

template <typename T>
struct Edge {
    T dx, dy, dz, r, g, dg, id;   // d = x_j - x_i, |d|, exp(gamma/(s-a)), dg/dr, 1/(s-a)
    int j;
};

template <typename T>
struct AdArgs {
    const double* x;     // SoA [3n]
    const double* w;     // SoA [3n] dual direction of x (NULL: zero)
    int n;
    double box[3];
    const int* nbr;
    const int* cnt;
    int cap;
    SWad<T> P;
    double* f;           // SoA [3n] forces (real part)
    double* fd;          // SoA [3n] dual part of the forces (NULL: not written)
    double* part;        // [gridDim.x][kRed] block partial sums
    unsigned* err;
};

// Minimum-image difference x_b - x_a along one axis (real part), dual part w_b - w_a.
template <typename T>
__device__ __forceinline__ T diff(const AdArgs<T>& A, int k, int a, int b) {
    const size_t N = (size_t)A.n;
    double d = A.x[k * N + b] - A.x[k * N + a];
    d -= A.box[k] * rint(d / A.box[k]);
    const double dd = A.w ? A.w[k * N + b] - A.w[k * N + a] : 0.0;
    return lift<T>(d, dd);
}

// Edge terms for d = x_j - x_i: false when |d| is at or beyond a*sigma (within 1e-12 sigma).
template <typename T>
__device__ __forceinline__ bool make_edge(const SWad<T>& P, T dx, T dy, T dz, int j, Edge<T>& e) {
    const double r2v = val(dx) * val(dx) + val(dy) * val(dy) + val(dz) * val(dz);
    if (!(r2v < P.rc2)) return false;
    const T r = f_sqrt(dx * dx + dy * dy + dz * dz);
    const T den = r * P.inv_sig - P.a;
    if (!(val(den) < -1e-12)) return false;
    e.dx = dx; e.dy = dy; e.dz = dz; e.r = r; e.j = j;
    e.id = f_rcp(den);
    e.g = f_exp(P.gam * e.id);
    e.dg = e.g * (-(P.gam * e.id * e.id)) * P.inv_sig;
    return true;
}

// Pair potential phi(r), dphi/dr and d phi / d(A, B, p, q, a).
template <typename T>
__device__ __forceinline__ void pair_terms(const SWad<T>& P, const Edge<T>& e, T& phi, T& dphi, T pg[5]) {
    const T s = e.r * P.inv_sig;
    const T e1 = f_exp(e.id);
    const T ls = f_log(s);
    const T rp = f_exp(-(P.p * ls)), rq = f_exp(-(P.q * ls));
    const T ea = P.eps * (P.A * e1);
    const T br = P.B * rp - rq;
    phi = ea * br;
    const T is = f_rcp(s);
    const T dphids = ea * ((P.q * rq - P.p * (P.B * rp)) * is) - phi * (e.id * e.id);
    dphi = dphids * P.inv_sig;
    pg[0] = P.eps * e1 * br;
    pg[1] = ea * rp;
    pg[2] = -(ea * (P.B * rp) * ls);
    pg[3] = ea * rq * ls;
    pg[4] = phi * (e.id * e.id);
}

// Triplet h(d1, d2) centred on the common atom: value and gradients with respect to the two
// leg vectors (d = leg atom - centre).
template <typename T>
__device__ __forceinline__ T triplet(const SWad<T>& P, const Edge<T>& a, const Edge<T>& b,
                                     T ga[3], T gb[3], T& dc_out) {
    const T ira = f_rcp(a.r), irb = f_rcp(b.r);
    const T c = (a.dx * b.dx + a.dy * b.dy + a.dz * b.dz) * ira * irb;
    const T dc = c - P.c0;
    const T el = P.eps * P.lam;
    const T hdc = el * dc * dc;
    // dh/dd_a = 2 el dc g_a g_b (d_b/(r_a r_b) - c d_a/r_a^2) + el dc^2 g_b (dg/dr)_a d_a/r_a
    const T tw = 2.0 * (el * dc * a.g * b.g);
    const T qq = tw * ira * irb;
    const T ka = hdc * a.dg * b.g * ira - tw * c * ira * ira;
    const T kb = hdc * a.g * b.dg * irb - tw * c * irb * irb;
    ga[0] = qq * b.dx + ka * a.dx; ga[1] = qq * b.dy + ka * a.dy; ga[2] = qq * b.dz + ka * a.dz;
    gb[0] = qq * a.dx + kb * b.dx; gb[1] = qq * a.dy + kb * b.dy; gb[2] = qq * a.dz + kb * b.dz;
    dc_out = dc;
    return hdc * a.g * b.g;
}

template <typename T>
__device__ __forceinline__ void warp_block_sum(double (&v)[kRed], double* out_block) {
    __shared__ double red[kAdThreads / 32][kRed];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < kRed; ++k) {
        double x = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) red[w][k] = x;
    }
    __syncthreads();
    if (threadIdx.x < kRed) {
        double s = 0.0;
        for (int i = 0; i < kAdThreads / 32; ++i) s += red[i][threadIdx.x];
        out_block[threadIdx.x] = s;
    }
}

// One thread per atom.  T = double: energy, forces and dU/dtheta; T = Dd: also their dual parts.
template <typename T>
__global__ void __launch_bounds__(kAdThreads) k_sw_ad(AdArgs<T> A) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const SWad<T>& P = A.P;
    T fx = lift<T>(0, 0), fy = fx, fz = fx, en = fx;
    T pg[7] = {fx, fx, fx, fx, fx, fx, fx};
    if (i < A.n) {
        Edge<T> sh[kAdShell];
        int m = 0;
        const int ci = min(A.cnt[i], A.cap);
        const int* row = A.nbr + (size_t)i * A.cap;
        for (int t = 0; t < ci; ++t) {
            const int j = row[t] & (int)kIndexMask;
            Edge<T> e;
            if (make_edge(P, diff(A, 0, i, j), diff(A, 1, i, j), diff(A, 2, i, j), j, e)) {
                if (m < kAdShell) sh[m] = e;
                ++m;
            }
        }
        if (m > kAdShell) {
            atomicOr(A.err, NEFE_ERR_SHELL_OVERFLOW);
            m = kAdShell;
        }
        // pair terms: full force on i, half the energy and parameter derivatives
        for (int t = 0; t < m; ++t) {
            T phi, dphi, pp[5];
            pair_terms(P, sh[t], phi, dphi, pp);
            const T c = dphi * f_rcp(sh[t].r);
            fx += c * sh[t].dx; fy += c * sh[t].dy; fz += c * sh[t].dz;
            en += 0.5 * phi;
            for (int k = 0; k < 5; ++k) pg[k] += 0.5 * pp[k];
        }
        // triplets centred on i
        for (int a = 0; a < m; ++a) {
            for (int b = a + 1; b < m; ++b) {
                T ga[3], gb[3], dc;
                const T h = triplet(P, sh[a], sh[b], ga, gb, dc);
                fx += ga[0] + gb[0]; fy += ga[1] + gb[1]; fz += ga[2] + gb[2];
                en += h;
                pg[4] += h * P.gam * (sh[a].id * sh[a].id + sh[b].id * sh[b].id);
                pg[5] += P.eps * dc * dc * sh[a].g * sh[b].g;
                pg[6] += h * (sh[a].id + sh[b].id);
            }
        }
        // triplets centred on each neighbour j in which i is a leg
        for (int a = 0; a < m; ++a) {
            const int j = sh[a].j;
            Edge<T> ij;                 // leg j -> i
            ij.dx = -sh[a].dx; ij.dy = -sh[a].dy; ij.dz = -sh[a].dz;
            ij.r = sh[a].r; ij.g = sh[a].g; ij.dg = sh[a].dg; ij.id = sh[a].id; ij.j = i;
            const int cj = min(A.cnt[j], A.cap);
            const int* rowj = A.nbr + (size_t)j * A.cap;
            for (int t = 0; t < cj; ++t) {
                const int k = rowj[t] & (int)kIndexMask;
                if (k == i) continue;
                Edge<T> jk;
                if (!make_edge(P, diff(A, 0, j, k), diff(A, 1, j, k), diff(A, 2, j, k), k, jk)) continue;
                T ga[3], gb[3], dc;
                triplet(P, ij, jk, ga, gb, dc);
                fx -= ga[0]; fy -= ga[1]; fz -= ga[2];
            }
        }
        const size_t N = (size_t)A.n;
        A.f[i] = val(fx); A.f[N + i] = val(fy); A.f[2 * N + i] = val(fz);
        if (A.fd) { A.fd[i] = dua(fx); A.fd[N + i] = dua(fy); A.fd[2 * N + i] = dua(fz); }
        if (!(isfinite(val(en)) && isfinite(val(fx)) && isfinite(val(fy)) && isfinite(val(fz))))
            atomicOr(A.err, NEFE_ERR_NAN);
    }
    double red[kRed];
    red[0] = val(en); red[1] = dua(en);
    for (int k = 0; k < 7; ++k) { red[2 + k] = val(pg[k]); red[9 + k] = dua(pg[k]); }
    warp_block_sum<T>(red, A.part + (size_t)blockIdx.x * kRed);
}

// Sums nb rows of width kRed in a fixed order (one warp per column).
__global__ void k_sum_rows(const double* part, int nb, int width, double* out) {
    const int c = blockIdx.x;
    double s = 0.0;
    for (int b = threadIdx.x; b < nb; b += 32) s += part[(size_t)b * width + c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) out[c] = s;
}

SWad<double> params_real(const nefe_sw_params& p) {
    SWad<double> c;
    c.eps = p.eps; c.inv_sig = 1.0 / p.sigma; c.c0 = p.cos0;
    const double rc = p.a * p.sigma;
    c.rc2 = rc * rc;
    c.A = p.A; c.B = p.B; c.p = p.p; c.q = p.q; c.a = p.a; c.lam = p.lambda3; c.gam = p.gamma;
    return c;
}

SWad<Dd> params_dual(const nefe_sw_params& p, const double* dth) {
    SWad<Dd> c;
    const double z[7] = {0, 0, 0, 0, 0, 0, 0};
    const double* d = dth ? dth : z;
    c.eps = p.eps; c.inv_sig = 1.0 / p.sigma; c.c0 = p.cos0;
    const double rc = p.a * p.sigma;
    c.rc2 = rc * rc;
    c.A = mk(p.A, d[0]); c.B = mk(p.B, d[1]); c.p = mk(p.p, d[2]); c.q = mk(p.q, d[3]);
    c.a = mk(p.a, d[4]); c.lam = mk(p.lambda3, d[5]); c.gam = mk(p.gamma, d[6]);
    return c;
}

inline int ad_blocks(int n) { return (n + kAdThreads - 1) / kAdThreads; }

// Launches the SW evaluation; out16 receives [E, E', G(7), G'(7)].
void launch_sw_ad(const double* x, const double* w, int n, const double box[3], const int* nbr,
                  const int* cnt, int cap, const nefe_sw_params& prm, const double* dth, bool dual,
                  double* f, double* fd, double* part, double* out16, unsigned* err, cudaStream_t s) {
    const int nb = ad_blocks(n);
    if (nb > 0) {
        if (dual) {
            AdArgs<Dd> A;
            A.x = x; A.w = w; A.n = n; A.nbr = nbr; A.cnt = cnt; A.cap = cap;
            for (int k = 0; k < 3; ++k) A.box[k] = box[k];
            A.P = params_dual(prm, dth); A.f = f; A.fd = fd; A.part = part; A.err = err;
            k_sw_ad<Dd><<<nb, kAdThreads, 0, s>>>(A);
        } else {
            AdArgs<double> A;
            A.x = x; A.w = nullptr; A.n = n; A.nbr = nbr; A.cnt = cnt; A.cap = cap;
            for (int k = 0; k < 3; ++k) A.box[k] = box[k];
            A.P = params_real(prm); A.f = f; A.fd = fd; A.part = part; A.err = err;
            k_sw_ad<double><<<nb, kAdThreads, 0, s>>>(A);
        }
        k_sum_rows<<<kRed, 32, 0, s>>>(part, nb, kRed, out16);
    } else {
        cudaMemsetAsync(out16, 0, sizeof(double) * kRed, s);
    }
}

// ---------------------------------------------------------------------------- integrator parts
// Per-step constants of the update, in FP64.
struct StepC {
    double c;      // dt / (2 m)
    double dt;
    double gm;     // m / tdamp (0 without thermostat)
    double amp;    // sqrt(2 m kB T / (tdamp dt)) (0 without thermostat)
    double kE;
    double s_int, s_E;   // force scales at the step's lambda
    double inv_n;
};

// vh = v + c F; x += dt vh (and the same for the tangents when X != NULL).
__global__ void k_half_drift(int n3, StepC C, double* x, const double* v, const double* F, double* vh,
                             double* X, const double* V, const double* Fd, double* VH) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n3) return;
    const double h = v[t] + C.c * F[t];
    vh[t] = h;
    x[t] = x[t] + C.dt * h;
    if (X) {
        const double H = V[t] + C.c * Fd[t];
        VH[t] = H;
        X[t] = X[t] + C.dt * H;
    }
}

// Per-block sums of the noise (3 components), of |x - r0|^2 and of (x - r0) . X.
__global__ void __launch_bounds__(kAdThreads) k_noise_spring_part(int n, const double* xi_aos, const double* x,
                                                                  const double* r0, const double* X, double* part) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double v[kRed];
    for (int k = 0; k < kRed; ++k) v[k] = 0.0;
    if (i < n) {
        const size_t N = (size_t)n;
        for (int k = 0; k < 3; ++k) {
            if (xi_aos) v[k] = xi_aos[3 * i + k];
            if (r0) {
                const double d = x[k * N + i] - r0[k * N + i];
                v[3] += d * d;
                if (X) v[4] += d * X[k * N + i];
            }
        }
    }
    warp_block_sum<double>(v, part + (size_t)blockIdx.x * kRed);
}

// F = s_int F_sw + s_E (-kE (x - r0)) - gm vh + amp (xi - mean xi); v = vh + c F (and the tangents).
__global__ void k_finish(int n, StepC C, const double* fsw, const double* x, const double* r0, const double* vh,
                         const double* xi_aos, const double* sums, double* F, double* v,
                         const double* fswd, const double* X, const double* VH, double* Fd, double* V) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 3 * n) return;
    const int k = t / n, i = t - k * n;
    double f = C.s_int * fsw[t] - C.gm * vh[t];
    if (r0 && C.s_E != 0.0) f -= C.s_E * C.kE * (x[t] - r0[t]);
    if (xi_aos) f += C.amp * (xi_aos[3 * i + k] - sums[k] * C.inv_n);
    F[t] = f;
    v[t] = vh[t] + C.c * f;
    if (Fd) {
        double g = C.s_int * fswd[t] - C.gm * VH[t];
        if (r0 && C.s_E != 0.0) g -= C.s_E * C.kE * X[t];
        Fd[t] = g;
        V[t] = VH[t] + C.c * g;
    }
}

// Work scalars on the device.
struct Scal {
    double sw[kRed];     // last SW evaluation [E, E', G(7), G'(7)]
    double ns[kRed];     // last noise / spring sums
    double W, dW;
    double th[7];        // accumulated dW/dtheta (reverse sweep)
};

// W += D dl with D = U_E - U (FL) or U + P V (RS); dW += D' dl.
__global__ void k_work(Scal* S, int kind, double kE, double PV, double dl) {
    const double ue = 0.5 * kE * S->ns[3], ued = kE * S->ns[4];
    double D, Dd_;
    if (kind == NEFE_SCHED_FL) { D = ue - S->sw[0]; Dd_ = ued - S->sw[1]; }
    else { D = S->sw[0] + PV; Dd_ = S->sw[1]; }
    S->W += D * dl;
    S->dW += Dd_ * dl;
}

// Reverse sweep, before the evaluation at x_{k+1}: w = fb + c vb (adjoint of F_{k+1}).
__global__ void k_rev_pre(int n3, double c, const double* fb, const double* vb, double* w) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n3) w[t] = fb[t] + c * vb[t];
}

// Reverse sweep after the evaluation at x_{k+1} (fsw, fswd = J w there):
//   xb += s_int J w - s_E kE w + dl grad_x D(x_{k+1});  vh_b = vb - gm w + dt xb;  vb = vh_b;  fb = c vh_b.
// With final != 0 (the evaluation at x_0) it writes dW/dx0 into xb and dW/dv0 into vb instead.
__global__ void k_rev_post(int n3, StepC C, int kind, double dl, const double* x, const double* r0,
                           const double* fsw, const double* fswd, const double* w, double* xb, double* vb,
                           double* fb, int final_) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n3) return;
    double gD;
    if (kind == NEFE_SCHED_FL) gD = (r0 ? C.kE * (x[t] - r0[t]) : 0.0) + fsw[t];
    else gD = -fsw[t];
    double xbn = xb[t] + C.s_int * fswd[t] + dl * gD;
    if (r0 && C.s_E != 0.0) xbn -= C.s_E * C.kE * w[t];
    if (final_) {
        xb[t] = xbn;
        vb[t] = vb[t] - C.gm * w[t];
        return;
    }
    const double vh = vb[t] - C.gm * w[t] + C.dt * xbn;
    xb[t] = xbn;
    vb[t] = vh;
    fb[t] = C.c * vh;
}

// th += s_int (dF/dtheta)^T w + dl dD/dtheta = -s_int G' + dl (-G for FL, +G for RS).
__global__ void k_rev_theta(Scal* S, int kind, double s_int, double dl) {
    const int k = threadIdx.x;
    if (k >= 7) return;
    const double G = S->sw[2 + k], Gd = S->sw[9 + k];
    S->th[k] += -s_int * Gd + dl * (kind == NEFE_SCHED_FL ? -G : G);
}

inline int eblocks(long n) { return (int)((n + 255) / 256); }

}  // namespace ad
}  // namespace nefe

using namespace nefe;
using namespace nefe::ad;

// ---------------------------------------------------------------------------- adjoint context
struct nefe_adj {
    int device = 0;
    cudaStream_t s = nullptr;
    nefe_adjoint_desc d;
    nefe_sw_params prm;
    int n = 0;
    double rcs = 0;
    double PV = 0;
    long nsteps = 0;          // length of the last forward run
    std::vector<double> lam;  // lambda_0 .. lambda_K
    Scratch1 L;               // list-build scratch
    Bufs lb;
    // device arrays (SoA [3n] unless noted)
    double *x0 = nullptr, *v0 = nullptr, *r0 = nullptr;
    double *x = nullptr, *v = nullptr, *F = nullptr, *vh = nullptr, *fsw = nullptr, *fswd = nullptr;
    double *X = nullptr, *V = nullptr, *Fd = nullptr, *VH = nullptr;
    double *xb = nullptr, *vb = nullptr, *fb = nullptr, *w = nullptr;
    double* xi = nullptr;     // AoS [n][3] noise of one step
    double* part = nullptr;   // [nblocks][kRed]
    double* ckpt = nullptr;   // [nckpt][3][3n]: x, v, F
    double* seg = nullptr;    // [K_c][3n] positions x_{k+1} of one segment
    long nckpt = 0;
    int* nbr = nullptr;
    int* cnt = nullptr;
    Scal* S = nullptr;
    unsigned* err = nullptr;
    std::vector<void*> owned;

    template <typename P>
    cudaError_t alloc(P** p, size_t bytes) {
        void* q = nullptr;
        cudaError_t e = cudaMalloc(&q, bytes < 16 ? 16 : bytes);
        if (e == cudaSuccess) owned.push_back(q);
        *p = static_cast<P*>(q);
        return e;
    }
    ~nefe_adj() {
        for (void* p : owned) cudaFree(p);
    }
};

namespace {

double sched_lambda_host(const nefe_adjoint_desc& d, long k) {
    double tau = d.nsched > 0 ? (double)k / (double)d.nsched : 1.0;
    if (tau > 1.0) tau = 1.0;
    if (d.direction < 0) tau = 1.0 - tau;
    if (d.kind == NEFE_SCHED_FL) {
        const double t2 = tau * tau, t4 = t2 * t2;
        return tau * t4 * (70.0 * t4 - 315.0 * t2 * tau + 540.0 * t2 - 420.0 * tau + 126.0);
    }
    return 1.0 / (1.0 + tau * (1.0 / d.lambda_f - 1.0));
}

StepC step_consts(const nefe_adj* A, long k) {
    StepC C;
    const double me = A->d.mass * kMvv2e;
    C.c = 0.5 * A->d.dt / me;
    C.dt = A->d.dt;
    const bool th = A->d.tdamp > 0.0;
    C.gm = th ? me / A->d.tdamp : 0.0;
    C.amp = th ? std::sqrt(2.0 * me * kB * A->d.T / (A->d.tdamp * A->d.dt)) : 0.0;
    C.kE = A->d.k_E;
    const double l = A->lam[(size_t)k];
    if (A->d.kind == NEFE_SCHED_FL) { C.s_int = 1.0 - l; C.s_E = l; }
    else { C.s_int = l; C.s_E = 0.0; }
    C.inv_n = 1.0 / (double)A->n;
    return C;
}

int list_at(nefe_adj* A, const double* x) {
    A->lb.x = const_cast<double*>(x);
    launch_cells_and_list(A->lb, NEFE_FP32, (A->n + kTile - 1) / kTile, 1, 1, A->s, nullptr);
    return NEFE_OK;
}

// SW evaluation at x (list rebuilt there); dual with direction w (and dth) when dual.
void eval_at(nefe_adj* A, const double* x, const double* w, const double* dth, bool dual) {
    list_at(A, x);
    launch_sw_ad(x, w, A->n, A->d.box, A->nbr, A->cnt, A->d.nbr_cap, A->prm, dth, dual, A->fsw,
                 dual ? A->fswd : nullptr, A->part, A->S->sw, A->err, A->s);
}

// Noise of step `step` and spring sums at x; then F, v (and tangents) by k_finish.
void finish_at(nefe_adj* A, long step, const double* vsrc_half, bool tangent) {
    const int n = A->n;
    const bool th = A->d.tdamp > 0.0;
    if (th) launch_noise(A->d.seed, A->d.sys_id, (unsigned long long)step, n, NEFE_FP64, A->xi, A->s);
    const int nb = ad_blocks(n);
    k_noise_spring_part<<<nb, kAdThreads, 0, A->s>>>(n, th ? A->xi : nullptr, A->x, A->r0,
                                                       tangent ? A->X : nullptr, A->part);
    k_sum_rows<<<kRed, 32, 0, A->s>>>(A->part, nb, kRed, A->S->ns);
    const StepC C = step_consts(A, step);
    k_finish<<<eblocks(3L * n), 256, 0, A->s>>>(n, C, A->fsw, A->x, A->r0, vsrc_half, th ? A->xi : nullptr,
                                                A->S->ns, A->F, A->v, tangent ? A->fswd : nullptr,
                                                tangent ? A->X : nullptr, tangent ? A->VH : nullptr,
                                                tangent ? A->Fd : nullptr, tangent ? A->V : nullptr);
}

void work_at(nefe_adj* A, long k) {
    if (k >= A->nsteps) return;
    const double dl = A->lam[(size_t)k + 1] - A->lam[(size_t)k];
    k_work<<<1, 1, 0, A->s>>>(A->S, A->d.kind, A->d.k_E, A->PV, dl);
}

// Initial force at step 0 (damping on v0, noise with step counter 0), from x = x0, v = v0.
void setup_run(nefe_adj* A, bool tangent, const double* dth) {
    const size_t b3 = sizeof(double) * 3 * (size_t)A->n;
    cudaMemcpyAsync(A->x, A->x0, b3, cudaMemcpyDeviceToDevice, A->s);
    cudaMemcpyAsync(A->vh, A->v0, b3, cudaMemcpyDeviceToDevice, A->s);
    if (tangent) cudaMemcpyAsync(A->VH, A->V, b3, cudaMemcpyDeviceToDevice, A->s);
    eval_at(A, A->x, tangent ? A->X : nullptr, dth, tangent);
    finish_at(A, 0, A->vh, tangent);
    // finish_at wrote v = vh + c F; the state after setup keeps v = v0
    cudaMemcpyAsync(A->v, A->v0, b3, cudaMemcpyDeviceToDevice, A->s);
    if (tangent) cudaMemcpyAsync(A->V, A->VH, b3, cudaMemcpyDeviceToDevice, A->s);
    work_at(A, 0);
}

// One step k -> k+1 of the trajectory (and of the tangents).
void step_run(nefe_adj* A, long k, bool tangent, const double* dth) {
    const int n3 = 3 * A->n;
    const StepC C = step_consts(A, k);
    k_half_drift<<<eblocks(n3), 256, 0, A->s>>>(n3, C, A->x, A->v, A->F, A->vh, tangent ? A->X : nullptr,
                                                tangent ? A->V : nullptr, tangent ? A->Fd : nullptr,
                                                tangent ? A->VH : nullptr);
    eval_at(A, A->x, tangent ? A->X : nullptr, dth, tangent);
    finish_at(A, k + 1, A->vh, tangent);
    work_at(A, k + 1);
}

int read_errors(nefe_adj* A, const char* where) {
    unsigned e1 = 0;
    DevState st;
    NEFE_CU(cudaMemcpyAsync(&e1, A->err, sizeof(unsigned), cudaMemcpyDeviceToHost, A->s));
    NEFE_CU(cudaMemcpyAsync(&st, A->L.st, sizeof(st), cudaMemcpyDeviceToHost, A->s));
    NEFE_CU(cudaStreamSynchronize(A->s));
    NEFE_CU(cudaGetLastError());
    const unsigned e = e1 | st.err;
    if (e & NEFE_ERR_NBR_OVERFLOW) return fail(NEFE_EOVERFLOW, "%s: neighbour row above cap", where);
    if (e & NEFE_ERR_SHELL_OVERFLOW) return fail(NEFE_EOVERFLOW, "%s: shell above 32 neighbours", where);
    if (e & NEFE_ERR_NAN) return fail(NEFE_ENAN, "%s: non-finite energy or force", where);
    if (e) return fail(NEFE_EINVAL, "%s: error word 0x%x", where, e);
    return NEFE_OK;
}

int reset_errors(nefe_adj* A) {
    NEFE_CU(cudaMemsetAsync(A->err, 0, sizeof(unsigned), A->s));
    NEFE_CU(cudaMemsetAsync(reinterpret_cast<char*>(A->L.st) + offsetof(DevState, err), 0, sizeof(unsigned), A->s));
    return NEFE_OK;
}

int prepare_schedule(nefe_adj* A, long nsteps) {
    int rc = reset_errors(A);
    if (rc) return rc;
    A->nsteps = nsteps;
    A->lam.resize((size_t)nsteps + 1);
    for (long k = 0; k <= nsteps; ++k) A->lam[(size_t)k] = sched_lambda_host(A->d, k);
    const long kc = A->d.checkpoint_every;
    const long need = nsteps / kc + 1;
    if (need > A->nckpt) {
        if (A->ckpt) {
            NEFE_CU(cudaStreamSynchronize(A->s));
            for (auto it = A->owned.begin(); it != A->owned.end(); ++it)
                if (*it == A->ckpt) { A->owned.erase(it); break; }
            cudaFree(A->ckpt);
            A->ckpt = nullptr;
        }
        NEFE_CU(A->alloc(&A->ckpt, sizeof(double) * 9 * (size_t)A->n * (size_t)need));
        A->nckpt = need;
    }
    return NEFE_OK;
}

void save_ckpt(nefe_adj* A, long idx) {
    const size_t b3 = sizeof(double) * 3 * (size_t)A->n;
    double* c = A->ckpt + (size_t)idx * 9 * (size_t)A->n;
    cudaMemcpyAsync(c, A->x, b3, cudaMemcpyDeviceToDevice, A->s);
    cudaMemcpyAsync(c + 3 * (size_t)A->n, A->v, b3, cudaMemcpyDeviceToDevice, A->s);
    cudaMemcpyAsync(c + 6 * (size_t)A->n, A->F, b3, cudaMemcpyDeviceToDevice, A->s);
}

void load_ckpt(nefe_adj* A, long idx) {
    const size_t b3 = sizeof(double) * 3 * (size_t)A->n;
    const double* c = A->ckpt + (size_t)idx * 9 * (size_t)A->n;
    cudaMemcpyAsync(A->x, c, b3, cudaMemcpyDeviceToDevice, A->s);
    cudaMemcpyAsync(A->v, c + 3 * (size_t)A->n, b3, cudaMemcpyDeviceToDevice, A->s);
    cudaMemcpyAsync(A->F, c + 6 * (size_t)A->n, b3, cudaMemcpyDeviceToDevice, A->s);
}

int upload_aos(nefe_adj* A, const double* host, double* dev) {
    const size_t b3 = sizeof(double) * 3 * (size_t)A->n;
    NEFE_CU(cudaMemcpyAsync(A->w, host, b3, cudaMemcpyHostToDevice, A->s));
    launch_aos_soa(A->w, dev, A->n, 1, A->s);
    return NEFE_OK;
}

int download_aos(nefe_adj* A, const double* dev, double* host) {
    const size_t b3 = sizeof(double) * 3 * (size_t)A->n;
    launch_aos_soa(dev, A->w, A->n, 0, A->s);
    NEFE_CU(cudaMemcpyAsync(host, A->w, b3, cudaMemcpyDeviceToHost, A->s));
    return NEFE_OK;
}

}  // namespace

extern "C" {

int nefe_sw_dual(const double* x, const double* w, int n, const double box[3], double rcs, const int* nbr,
                 const int* cnt, int cap, const nefe_sw_params* prm, const double* dtheta, double* f,
                 double* fd, double* out16, void* stream) {
    NvtxRange nvtx_("nefe_sw_dual");
    if (n < 0 || !box || cap < 1 || cap > kMaxCap || !valid_params(prm) || !out16 ||
        (n > 0 && (!x || !nbr || !cnt || !f || !fd)))
        return fail(NEFE_EINVAL, "nefe_sw_dual: bad argument");
    if (prm->a * prm->sigma > rcs) return fail(NEFE_EINVAL, "nefe_sw_dual: a*sigma above rcs");
    int rc = check_box(box, rcs);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    double* part = nullptr;
    unsigned* err = nullptr;
    const int nb = ad_blocks(n);
    NEFE_CU(cudaMallocAsync(&part, sizeof(double) * kRed * (size_t)(nb > 0 ? nb : 1), s));
    NEFE_CU(cudaMallocAsync(&err, sizeof(unsigned), s));
    NEFE_CU(cudaMemsetAsync(err, 0, sizeof(unsigned), s));
    launch_sw_ad(x, w, n, box, nbr, cnt, cap, *prm, dtheta, true, f, fd, part, out16, err, s);
    unsigned e = 0;
    NEFE_CU(cudaMemcpyAsync(&e, err, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    cudaFreeAsync(part, s);
    cudaFreeAsync(err, s);
    NEFE_CU(cudaStreamSynchronize(s));
    NEFE_CU(cudaGetLastError());
    if (e & NEFE_ERR_SHELL_OVERFLOW) return fail(NEFE_EOVERFLOW, "nefe_sw_dual: shell above 32 neighbours");
    if (e & NEFE_ERR_NAN) return fail(NEFE_ENAN, "nefe_sw_dual: non-finite energy or force");
    return NEFE_OK;
}

int nefe_adjoint_create(nefe_adj** out, int device, void* stream, const nefe_adjoint_desc* d,
                        const nefe_sw_params* prm) {
    if (!out || !d || !valid_params(prm) || d->n <= 0 || !d->x || !d->v || d->mass <= 0 || d->dt <= 0 ||
        d->nbr_cap < 1 || d->nbr_cap > kMaxCap || d->checkpoint_every < 1 || d->skin < 0 ||
        (d->kind != NEFE_SCHED_FL && d->kind != NEFE_SCHED_RS) || (d->direction != 1 && d->direction != -1) ||
        d->nsched < 1 || (d->kind == NEFE_SCHED_FL && (!d->r0 || d->k_E <= 0)) ||
        (d->kind == NEFE_SCHED_RS && !(d->lambda_f > 0)) || (d->tdamp > 0 && !(d->T > 0)))
        return fail(NEFE_EINVAL, "nefe_adjoint_create: bad argument");
    if (d->n >= (1 << kCodeShift)) return fail(NEFE_EINVAL, "nefe_adjoint_create: n above 2^27");
    *out = nullptr;
    NEFE_CU(cudaSetDevice(device));
    const double rcs = prm->a * prm->sigma + d->skin;
    int rc = check_box(d->box, rcs);
    if (rc) return rc;
    int n3[3];
    if (!host_grid(d->box, rcs, n3)) return fail(NEFE_EINVAL, "nefe_adjoint_create: fewer than 2 cells on an axis");
    const long long total = (long long)n3[0] * n3[1] * n3[2];
    nefe_adj* A = new nefe_adj();
    A->device = device;
    A->s = (cudaStream_t)stream;
    A->d = *d;
    A->prm = *prm;
    A->n = d->n;
    A->rcs = rcs;
    A->PV = d->P_GPa / kEvA3ToGPa * d->box[0] * d->box[1] * d->box[2];
    A->L.s = A->s;
    const int n = A->n;
    const size_t b3 = sizeof(double) * 3 * (size_t)n;
    auto bail = [&](int code) { cudaStreamSynchronize(A->s); delete A; return code; };
    if ((rc = prepare1(A->L, n, d->box, rcs, (int)total, NEFE_FP32, true))) return bail(rc);
    A->lb = bufs_of(A->L, nullptr, n);
    double** arrs[] = {&A->x0, &A->v0, &A->x, &A->v, &A->F, &A->vh, &A->fsw, &A->fswd, &A->X, &A->V, &A->Fd,
                       &A->VH, &A->xb, &A->vb, &A->fb, &A->w, &A->xi};
    for (double** p : arrs)
        if (A->alloc(p, b3) != cudaSuccess) return bail(fail(NEFE_ENOMEM, "nefe_adjoint_create: device memory"));
    if (d->r0 && A->alloc(&A->r0, b3) != cudaSuccess) return bail(fail(NEFE_ENOMEM, "nefe_adjoint_create: r0"));
    if (A->alloc(&A->part, sizeof(double) * kRed * (size_t)ad_blocks(n)) != cudaSuccess ||
        A->alloc(&A->seg, b3 * (size_t)d->checkpoint_every) != cudaSuccess ||
        A->alloc(&A->nbr, sizeof(int) * (size_t)n * d->nbr_cap) != cudaSuccess ||
        A->alloc(&A->cnt, sizeof(int) * (size_t)n) != cudaSuccess ||
        A->alloc(&A->S, sizeof(Scal)) != cudaSuccess || A->alloc(&A->err, sizeof(unsigned)) != cudaSuccess)
        return bail(fail(NEFE_ENOMEM, "nefe_adjoint_create: device memory"));
    A->lb.nbr = A->nbr; A->lb.cnt = A->cnt; A->lb.cap = d->nbr_cap;
    if ((rc = upload_aos(A, d->x, A->x0)) || (rc = upload_aos(A, d->v, A->v0))) return bail(rc);
    if (d->r0 && (rc = upload_aos(A, d->r0, A->r0))) return bail(rc);
    if (cudaMemsetAsync(A->err, 0, sizeof(unsigned), A->s) != cudaSuccess ||
        cudaMemsetAsync(A->S, 0, sizeof(Scal), A->s) != cudaSuccess ||
        cudaStreamSynchronize(A->s) != cudaSuccess)
        return bail(cuda_fail(cudaGetLastError(), "nefe_adjoint_create"));
    A->d.x = A->d.v = A->d.r0 = nullptr;   // host arrays are not kept
    *out = A;
    return NEFE_OK;
}

int nefe_adjoint_set_params(nefe_adj* A, const nefe_sw_params* prm) {
    if (!A || !valid_params(prm)) return fail(NEFE_EINVAL, "nefe_adjoint_set_params: bad argument");
    if (prm->a * prm->sigma > A->rcs)
        return fail(NEFE_EINVAL, "nefe_adjoint_set_params: a*sigma above the list radius %g", A->rcs);
    A->prm = *prm;
    A->nsteps = 0;   // checkpoints belong to the old parameters
    return NEFE_OK;
}

int nefe_adjoint_destroy(nefe_adj* A) {
    if (!A) return NEFE_OK;
    cudaSetDevice(A->device);
    cudaStreamSynchronize(A->s);
    delete A;
    return NEFE_OK;
}

int nefe_adjoint_forward(nefe_adj* A, long nsteps, double* W) {
    NvtxRange nvtx_("nefe_adjoint_forward");
    if (!A || nsteps < 1) return fail(NEFE_EINVAL, "nefe_adjoint_forward: bad argument");
    NEFE_CU(cudaSetDevice(A->device));
    int rc = prepare_schedule(A, nsteps);
    if (rc) return rc;
    NEFE_CU(cudaMemsetAsync(A->S, 0, sizeof(Scal), A->s));
    setup_run(A, false, nullptr);
    save_ckpt(A, 0);
    const long kc = A->d.checkpoint_every;
    for (long k = 0; k < nsteps; ++k) {
        step_run(A, k, false, nullptr);
        if ((k + 1) % kc == 0 && k + 1 < nsteps) save_ckpt(A, (k + 1) / kc);
    }
    Scal h;
    NEFE_CU(cudaMemcpyAsync(&h, A->S, sizeof(h), cudaMemcpyDeviceToHost, A->s));
    rc = read_errors(A, "nefe_adjoint_forward");
    if (rc) return rc;
    if (W) *W = h.W;
    return NEFE_OK;
}

int nefe_adjoint_backward(nefe_adj* A, double dW_dtheta[7], double* dW_dx0, double* dW_dv0) {
    NvtxRange nvtx_("nefe_adjoint_backward");
    if (!A || !dW_dtheta) return fail(NEFE_EINVAL, "nefe_adjoint_backward: bad argument");
    if (A->nsteps < 1) return fail(NEFE_ESTATE, "nefe_adjoint_backward: run nefe_adjoint_forward first");
    NEFE_CU(cudaSetDevice(A->device));
    const int n = A->n, n3 = 3 * n;
    const size_t b3 = sizeof(double) * (size_t)n3;
    const long K = A->nsteps, kc = A->d.checkpoint_every;
    int rc0 = reset_errors(A);
    if (rc0) return rc0;
    NEFE_CU(cudaMemsetAsync(A->xb, 0, b3, A->s));
    NEFE_CU(cudaMemsetAsync(A->vb, 0, b3, A->s));
    NEFE_CU(cudaMemsetAsync(A->fb, 0, b3, A->s));
    NEFE_CU(cudaMemsetAsync(A->S->th, 0, sizeof(double) * 7, A->s));
    const long nseg = (K + kc - 1) / kc;
    for (long sg = nseg - 1; sg >= 0; --sg) {
        const long k0 = sg * kc, k1 = (k0 + kc < K) ? k0 + kc : K;
        // recompute the segment from its checkpoint, keeping x_{k+1}
        load_ckpt(A, sg);
        for (long k = k0; k < k1; ++k) {
            const StepC C = step_consts(A, k);
            k_half_drift<<<eblocks(n3), 256, 0, A->s>>>(n3, C, A->x, A->v, A->F, A->vh, nullptr, nullptr,
                                                        nullptr, nullptr);
            if (k + 1 < k1) {
                eval_at(A, A->x, nullptr, nullptr, false);
                finish_at(A, k + 1, A->vh, false);
            }
            cudaMemcpyAsync(A->seg + (size_t)(k - k0) * n3, A->x, b3, cudaMemcpyDeviceToDevice, A->s);
        }
        // step the adjoint variables back through the segment
        for (long k = k1 - 1; k >= k0; --k) {
            const double* xk1 = A->seg + (size_t)(k - k0) * n3;
            const StepC C1 = step_consts(A, k + 1);
            const double dl = (k + 1 < K) ? A->lam[(size_t)k + 2] - A->lam[(size_t)k + 1] : 0.0;
            k_rev_pre<<<eblocks(n3), 256, 0, A->s>>>(n3, C1.c, A->fb, A->vb, A->w);
            eval_at(A, xk1, A->w, nullptr, true);
            k_rev_post<<<eblocks(n3), 256, 0, A->s>>>(n3, C1, A->d.kind, dl, xk1, A->r0, A->fsw, A->fswd, A->w,
                                                      A->xb, A->vb, A->fb, 0);
            k_rev_theta<<<1, 32, 0, A->s>>>(A->S, A->d.kind, C1.s_int, dl);
        }
    }
    // the initial force F_0 = F(x_0) - gm v_0 + noise, and the work term at x_0
    {
        const StepC C0 = step_consts(A, 0);
        const double dl = A->lam[1] - A->lam[0];
        NEFE_CU(cudaMemcpyAsync(A->w, A->fb, b3, cudaMemcpyDeviceToDevice, A->s));
        eval_at(A, A->x0, A->w, nullptr, true);
        k_rev_post<<<eblocks(n3), 256, 0, A->s>>>(n3, C0, A->d.kind, dl, A->x0, A->r0, A->fsw, A->fswd, A->w,
                                                  A->xb, A->vb, A->fb, 1);
        k_rev_theta<<<1, 32, 0, A->s>>>(A->S, A->d.kind, C0.s_int, dl);
    }
    Scal h;
    NEFE_CU(cudaMemcpyAsync(&h, A->S, sizeof(h), cudaMemcpyDeviceToHost, A->s));
    int rc = 0;
    if (dW_dx0 && (rc = download_aos(A, A->xb, dW_dx0))) return rc;
    if (dW_dv0 && (rc = download_aos(A, A->vb, dW_dv0))) return rc;
    rc = read_errors(A, "nefe_adjoint_backward");
    if (rc) return rc;
    for (int k = 0; k < 7; ++k) dW_dtheta[k] = h.th[k];
    return NEFE_OK;
}

int nefe_adjoint_tangent(nefe_adj* A, long nsteps, const double dtheta[7], const double* dx0,
                         const double* dv0, double* W, double* dW) {
    NvtxRange nvtx_("nefe_adjoint_tangent");
    if (!A || nsteps < 1 || !dtheta) return fail(NEFE_EINVAL, "nefe_adjoint_tangent: bad argument");
    NEFE_CU(cudaSetDevice(A->device));
    const size_t b3 = sizeof(double) * 3 * (size_t)A->n;
    int rc = prepare_schedule(A, nsteps);
    if (rc) return rc;
    NEFE_CU(cudaMemsetAsync(A->S, 0, sizeof(Scal), A->s));
    if (dx0) { if ((rc = upload_aos(A, dx0, A->X))) return rc; }
    else NEFE_CU(cudaMemsetAsync(A->X, 0, b3, A->s));
    if (dv0) { if ((rc = upload_aos(A, dv0, A->V))) return rc; }
    else NEFE_CU(cudaMemsetAsync(A->V, 0, b3, A->s));
    setup_run(A, true, dtheta);
    for (long k = 0; k < nsteps; ++k) step_run(A, k, true, dtheta);
    Scal h;
    NEFE_CU(cudaMemcpyAsync(&h, A->S, sizeof(h), cudaMemcpyDeviceToHost, A->s));
    rc = read_errors(A, "nefe_adjoint_tangent");
    A->nsteps = 0;   // no checkpoints of this run: a backward needs a forward first
    if (rc) return rc;
    if (W) *W = h.W;
    if (dW) *dW = h.dW;
    return NEFE_OK;
}

int nefe_adjoint_state(nefe_adj* A, double* x, double* v) {
    if (!A) return fail(NEFE_EINVAL, "nefe_adjoint_state: bad argument");
    NEFE_CU(cudaSetDevice(A->device));
    int rc = 0;
    if (x && (rc = download_aos(A, A->x, x))) return rc;
    if (v && (rc = download_aos(A, A->v, v))) return rc;
    NEFE_CU(cudaStreamSynchronize(A->s));
    return NEFE_OK;
}

}  // extern "C"
