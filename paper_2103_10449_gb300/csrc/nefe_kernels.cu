// libnefe device kernels for sm_103a.
//
// Step sequence of one time step k -> k+1 (all systems of a context at once):
//   k_group       per system / dCCI pair: reads the fixed-point sums of step k, observes
//                 P, V, dH/dl, records, kicks the barostat, advances lambda and W (Eq. Wdyn,
//                 left point), applies the dCCI update (Eqs. Ps_coex_discreted /
//                 l_coex_discreted), sets this step's drift factors and zeroes the sums.
//   k_kick_drift  v += dt/2 F/m; x = s x + dt phi v (affine box drift); FP32/FP64 mirror
//                 xs = x - q h; displacement test -> rebuild flag; sum of thermostat noise.
//   rebuild       (flagged systems) cell count -> scan -> fill -> per-cell sort -> list.
//   k_force       SW pair + triplet gather (FP32 or FP64), Einstein springs (FP64), lambda
//                 mixing, Langevin force with its mean removed, second half kick, sums.
#include <cuda_runtime.h>
#include <stdint.h>

#include "nefe.h"
#include "nefe_dev.h"
#include "nefe_launch.h"

namespace nefe {

template <typename T> struct V4;
template <> struct V4<float> { using t = float4; };
template <> struct V4<double> { using t = double4; };

__device__ __forceinline__ float4 mk4(float a, float b, float c, float d) { return make_float4(a, b, c, d); }
__device__ __forceinline__ double4 mk4(double a, double b, double c, double d) { return make_double4(a, b, c, d); }

// ------------------------------------------------------------------------------------
// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11): round (hi0,lo0) = M0 X0,
// (hi1,lo1) = M1 X2, X <- (hi1^X1^k0, lo1, hi0^X3^k1, lo0), key += Weyl constants.
// ------------------------------------------------------------------------------------
__device__ __forceinline__ void philox4x64_10(uint64_t c[4], uint64_t k0, uint64_t k1) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t hi0 = __umul64hi(M0, c[0]), lo0 = M0 * c[0];
        const uint64_t hi1 = __umul64hi(M1, c[2]), lo1 = M1 * c[2];
        const uint64_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
        k0 += W0; k1 += W1;
    }
}

// Three standard normals for (seed, system, step, atom): counter (step, atom, system, 0),
// key (seed, 0); Box-Muller on the (0,1) uniforms of outputs (0,1) and (2,3).
template <typename T> struct Noise;
template <> struct Noise<double> {
    __device__ static void xi3(uint64_t seed, uint64_t sys, uint64_t step, uint64_t id, double out[3]) {
        uint64_t c[4] = {step, id, sys, 0ULL};
        philox4x64_10(c, seed, 0ULL);
        const double u0 = ((double)(c[0] >> 11) + 0.5) * 0x1p-53;
        const double u1 = ((double)(c[1] >> 11) + 0.5) * 0x1p-53;
        const double u2 = ((double)(c[2] >> 11) + 0.5) * 0x1p-53;
        const double u3 = ((double)(c[3] >> 11) + 0.5) * 0x1p-53;
        const double two_pi = 6.283185307179586476925286766559;
        const double r0 = sqrt(-2.0 * log(u0)), r1 = sqrt(-2.0 * log(u2));
        double s0, c0, s1, c1;
        sincos(two_pi * u1, &s0, &c0);
        sincos(two_pi * u3, &s1, &c1);
        out[0] = r0 * c0; out[1] = r0 * s0; out[2] = r1 * c1;
    }
};
template <> struct Noise<float> {
    __device__ static void xi3(uint64_t seed, uint64_t sys, uint64_t step, uint64_t id, float out[3]) {
        uint64_t c[4] = {step, id, sys, 0ULL};
        philox4x64_10(c, seed, 0ULL);
        const float u0 = ((float)(c[0] >> 40) + 0.5f) * 0x1p-24f;
        const float u1 = ((float)(c[1] >> 40) + 0.5f) * 0x1p-24f;
        const float u2 = ((float)(c[2] >> 40) + 0.5f) * 0x1p-24f;
        const float u3 = ((float)(c[3] >> 40) + 0.5f) * 0x1p-24f;
        const float r0 = sqrtf(-2.0f * logf(u0)), r1 = sqrtf(-2.0f * logf(u2));
        float s0, c0, s1, c1;
        sincospif(2.0f * u1, &s0, &c0);
        sincospif(2.0f * u3, &s1, &c1);
        out[0] = r0 * c0; out[1] = r0 * s0; out[2] = r1 * c1;
    }
};

// ------------------------------------------------------------------------------------
// Deterministic per-system sums: warp shuffle -> shared -> one int64 fixed-point atomic per
// value into slot (blockIdx % kSlots).  Every thread of the block must call it.
// ------------------------------------------------------------------------------------
template <typename T, int K>
__device__ __forceinline__ void block_sum_to_acc(T (&v)[K], long long* acc_sys, int first,
                                                 unsigned* err) {
    __shared__ double red[kTile / 32][K];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        T x = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) red[w][k] = (double)x;
    }
    __syncthreads();
    if (threadIdx.x < K) {
        double s = 0.0;
#pragma unroll
        for (int i = 0; i < kTile / 32; ++i) s += red[i][threadIdx.x];
        if (!isfinite(s)) {
            atomicOr(err, NEFE_ERR_NAN);
        } else if (s != 0.0) {
            const long long q = __double2ll_rn(s * kFix);
            atomicAdd(reinterpret_cast<unsigned long long*>(
                          &acc_sys[(size_t)(first + threadIdx.x) * kSlots + (blockIdx.x % kSlots)]),
                      (unsigned long long)q);
        }
    }
}

// Cell grid for a box: per axis floor(L/rcs), reduced while L/n < rcs (1 + 1e-9); then the
// largest axis is reduced until the product fits the capacity (wider cells stay valid).
__device__ __forceinline__ bool grid_for(const double box[3], double rcs, int cap, int n3[3]) {
    bool ok = true;
    for (int k = 0; k < 3; ++k) {
        int m = (int)floor(__ddiv_rn(box[k], rcs));
        while (m > 0 && __ddiv_rn(box[k], (double)m) < rcs * (1.0 + 1e-9)) --m;
        if (m < 2) { ok = false; m = 2; }
        n3[k] = m;
    }
    while ((long long)n3[0] * n3[1] * n3[2] > cap) {
        int k = (n3[0] >= n3[1] && n3[0] >= n3[2]) ? 0 : (n3[1] >= n3[2] ? 1 : 2);
        if (n3[k] <= 2) { ok = false; break; }
        --n3[k];
    }
    return ok;
}

struct TileAtom {
    int sys, first, count;
};
__device__ __forceinline__ TileAtom tile_of(const Bufs& b, int tile) {
    TileAtom t;
    t.sys = b.tile_sys[tile];
    const DevSys& S = b.sys[t.sys];
    t.first = S.off + (tile - S.tile0) * kTile;
    t.count = min(kTile, S.off + S.n - t.first);
    return t;
}

// ------------------------------------------------------------------------------------
// Rebuild: R1 cell of each atom, unwrapped cell index q, fresh mirror, occupancy count.
// The cell formula is c = (int)(w n) with w = x/L - floor(x/L) evaluated in FP64.
// ------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kTile) k_cells_count(Bufs b, int force_all) {
    using T4 = typename V4<T>::t;
    const TileAtom ta = tile_of(b, blockIdx.x);
    const DevSys& S = b.sys[ta.sys];
    DevState& st = b.st[ta.sys];
    if (!force_all && !st.rebuild) return;
    int n3[3];
    const bool ok = grid_for(st.box, S.rcs, S.ncell_cap, n3);
    double h[3];
    for (int k = 0; k < 3; ++k) h[k] = __ddiv_rn(st.box[k], (double)n3[k]);
    if (blockIdx.x == S.tile0 && threadIdx.x == 0) {
        for (int k = 0; k < 3; ++k) { st.ncell[k] = n3[k]; st.h[k] = h[k]; st.hb[k] = h[k]; }
        st.nbuild += 1;
        if (!ok) atomicOr(&st.err, NEFE_ERR_BOX);
    }
    if ((int)threadIdx.x >= ta.count) return;
    const int i = ta.first + threadIdx.x;
    int c3[3], qv[3];
    double xs[3];
    for (int k = 0; k < 3; ++k) {
        const double xk = b.x[(size_t)k * b.ntot + i];
        const double s = __ddiv_rn(xk, st.box[k]);
        const double fl = floor(s);
        const double w = __dsub_rn(s, fl);
        int c = (int)__dmul_rn(w, (double)n3[k]);
        if (c >= n3[k]) c = n3[k] - 1;
        if (c < 0) c = 0;
        c3[k] = c;
        qv[k] = (int)fl * n3[k] + c;
        xs[k] = xk - (double)qv[k] * h[k];
    }
    const int cell = c3[0] + n3[0] * (c3[1] + n3[1] * c3[2]);
    b.cell_of[i] = cell;
    b.q[i] = make_int4(qv[0], qv[1], qv[2], 0);
    const T4 m = mk4((T)xs[0], (T)xs[1], (T)xs[2], (T)0);
    reinterpret_cast<T4*>(b.xs)[i] = m;
    reinterpret_cast<T4*>(b.xsb)[i] = m;
    atomicAdd(&b.cell_count[S.cell0 + cell], 1);
}

// R2: exclusive scan of the occupancy (one 256-thread block per system); resets counts.
__global__ void __launch_bounds__(256) k_cells_scan(Bufs b, int force_all) {
    const int s = blockIdx.x;
    const DevSys& S = b.sys[s];
    DevState& st = b.st[s];
    if (!force_all && !st.rebuild) return;
    const int ncells = st.ncell[0] * st.ncell[1] * st.ncell[2];
    int* start = b.cell_start + S.cell0 + s;
    int* count = b.cell_count + S.cell0;
    int* cursor = b.cell_cursor + S.cell0;
    __shared__ int warp_tot[8];
    __shared__ int carry_s;
    if (threadIdx.x == 0) carry_s = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int base = 0; base < ncells; base += 256) {
        const int idx = base + threadIdx.x;
        const int c = idx < ncells ? count[idx] : 0;
        int incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) warp_tot[w] = incl;
        __syncthreads();
        int woff = 0, tot = 0;
        for (int k = 0; k < 8; ++k) {
            if (k < w) woff += warp_tot[k];
            tot += warp_tot[k];
        }
        const int carry = carry_s;
        if (idx < ncells) {
            const int excl = carry + woff + incl - c;
            start[idx] = excl;
            cursor[idx] = excl;
            count[idx] = 0;
        }
        __syncthreads();
        if (threadIdx.x == 0) carry_s = carry + tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) start[ncells] = carry_s;
}

// R3: scatter atoms into their cell segment (order inside a cell fixed by R4).
__global__ void __launch_bounds__(kTile) k_cells_fill(Bufs b, int force_all) {
    const TileAtom ta = tile_of(b, blockIdx.x);
    const DevSys& S = b.sys[ta.sys];
    if (!force_all && !b.st[ta.sys].rebuild) return;
    if ((int)threadIdx.x >= ta.count) return;
    const int i = ta.first + threadIdx.x;
    const int pos = atomicAdd(&b.cell_cursor[S.cell0 + b.cell_of[i]], 1);
    b.perm[S.off + pos] = i;
}

// R4: insertion sort of each cell segment by atom index (stable order by (cell, atom)).
__global__ void __launch_bounds__(256) k_cells_sort(Bufs b, int force_all) {
    const int s = blockIdx.x;
    const DevSys& S = b.sys[s];
    const DevState& st = b.st[s];
    if (!force_all && !st.rebuild) return;
    const int ncells = st.ncell[0] * st.ncell[1] * st.ncell[2];
    const int* start = b.cell_start + S.cell0 + s;
    int* p = b.perm + S.off;
    for (int c = threadIdx.x; c < ncells; c += blockDim.x) {
        const int lo = start[c], hi = start[c + 1];
        for (int a = lo + 1; a < hi; ++a) {
            const int key = p[a];
            int z = a - 1;
            while (z >= lo && p[z] > key) { p[z + 1] = p[z]; --z; }
            p[z + 1] = key;
        }
    }
}

// Exact list criterion in FP64, the plain definition: raw = x_j - x_i, m = rint(raw/L),
// d = raw - m L, ((d_x^2 + d_y^2) + d_z^2) < rcs^2; every operation rounded separately.
__device__ __forceinline__ bool exact_pair_in(const Bufs& b, const double box[3], int i, int j,
                                              double rcs2, double d[3]) {
    for (int k = 0; k < 3; ++k) {
        const double raw = __dsub_rn(b.x[(size_t)k * b.ntot + j], b.x[(size_t)k * b.ntot + i]);
        const double m = rint(__ddiv_rn(raw, box[k]));
        d[k] = __dsub_rn(raw, __dmul_rn(m, box[k]));
    }
    double rr = __dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1]));
    rr = __dadd_rn(rr, __dmul_rn(d[2], d[2]));
    return rr < rcs2;
}

// R5: Verlet list of atom i from the 27 cell offsets.  A candidate is accepted or rejected
// on its mirror distance when that is outside a relative band of 1e-4 (FP32) / 1e-10 (FP64)
// around rcs^2; inside the band the exact FP64 criterion decides (and must agree with the
// offset's image), so the list equals the plain definition bit for bit.
template <typename T>
__global__ void __launch_bounds__(kTile) k_nlist(Bufs b, int force_all) {
    using T4 = typename V4<T>::t;
    const TileAtom ta = tile_of(b, blockIdx.x);
    const DevSys& S = b.sys[ta.sys];
    DevState& st = b.st[ta.sys];
    if (!force_all && !st.rebuild) return;
    if ((int)threadIdx.x >= ta.count) return;
    const int i = ta.first + threadIdx.x;
    const int nx = st.ncell[0], ny = st.ncell[1], nz = st.ncell[2];
    const int cell = b.cell_of[i];
    const int cx = cell % nx, cy = (cell / nx) % ny, cz = cell / (nx * ny);
    const T4 xi = reinterpret_cast<const T4*>(b.xs)[i];
    const T hx = (T)st.h[0], hy = (T)st.h[1], hz = (T)st.h[2];
    const double rcs2 = __dmul_rn(S.rcs, S.rcs);
    const T band = sizeof(T) == 4 ? (T)1e-4 : (T)1e-10;
    const T lo2 = (T)rcs2 * ((T)1 - band), hi2 = (T)rcs2 * ((T)1 + band);
    const int* start = b.cell_start + S.cell0 + ta.sys;
    int row[kMaxCap];
    int count = 0;
    const int cap = b.cap;
    for (int oz = -1; oz <= 1; ++oz) {
        const int czz = (cz + oz + nz) % nz;
        for (int oy = -1; oy <= 1; ++oy) {
            const int cyy = (cy + oy + ny) % ny;
            for (int ox = -1; ox <= 1; ++ox) {
                const int cxx = (cx + ox + nx) % nx;
                const int c2 = cxx + nx * (cyy + ny * czz);
                const int code = (ox + 1) + 3 * (oy + 1) + 9 * (oz + 1);
                const int pe = start[c2 + 1];
                for (int p = start[c2]; p < pe; ++p) {
                    const int j = b.perm[S.off + p];
                    if (j == i && code == 13) continue;
                    const T4 xj = reinterpret_cast<const T4*>(b.xs)[j];
                    const T dx = xj.x - xi.x + (T)ox * hx;
                    const T dy = xj.y - xi.y + (T)oy * hy;
                    const T dz = xj.z - xi.z + (T)oz * hz;
                    const T dd = dx * dx + dy * dy + dz * dz;
                    bool in;
                    if (dd < lo2) {
                        in = true;
                    } else if (dd > hi2) {
                        in = false;
                    } else {
                        double d[3];
                        in = exact_pair_in(b, st.box, i, j, rcs2, d);
                        // the exact (minimum) image must be the one reached through this offset
                        in = in && fabs(d[0] - (double)dx) < 0.5 * st.h[0] &&
                             fabs(d[1] - (double)dy) < 0.5 * st.h[1] &&
                             fabs(d[2] - (double)dz) < 0.5 * st.h[2];
                    }
                    if (!in) continue;
                    if (count < cap) {
                        const int e = j | (code << kCodeShift);
                        int z = count;
                        while (z > 0 && (row[z - 1] & (int)kIndexMask) > j) { row[z] = row[z - 1]; --z; }
                        row[z] = e;
                    }
                    ++count;
                }
            }
        }
    }
    int* out = b.nbr + (size_t)i * cap;
    const int m = count < cap ? count : cap;
    for (int z = 0; z < m; ++z) out[z] = row[z];
    b.cnt[i] = count;
    if (count > cap) atomicOr(&st.err, NEFE_ERR_NBR_OVERFLOW);
}

// Mirror only (stateless forces): same q / xs formula as R1, without counting.
template <typename T>
__global__ void __launch_bounds__(kTile) k_mirror(Bufs b) {
    using T4 = typename V4<T>::t;
    const TileAtom ta = tile_of(b, blockIdx.x);
    const DevSys& S = b.sys[ta.sys];
    DevState& st = b.st[ta.sys];
    int n3[3];
    grid_for(st.box, S.rcs, S.ncell_cap, n3);
    double h[3];
    for (int k = 0; k < 3; ++k) h[k] = __ddiv_rn(st.box[k], (double)n3[k]);
    if (blockIdx.x == S.tile0 && threadIdx.x == 0)
        for (int k = 0; k < 3; ++k) { st.ncell[k] = n3[k]; st.h[k] = h[k]; st.hb[k] = h[k]; }
    if ((int)threadIdx.x >= ta.count) return;
    const int i = ta.first + threadIdx.x;
    double xs[3];
    for (int k = 0; k < 3; ++k) {
        const double xk = b.x[(size_t)k * b.ntot + i];
        const double s = __ddiv_rn(xk, st.box[k]);
        const double fl = floor(s);
        const double w = __dsub_rn(s, fl);
        int c = (int)__dmul_rn(w, (double)n3[k]);
        if (c >= n3[k]) c = n3[k] - 1;
        if (c < 0) c = 0;
        const int q = (int)fl * n3[k] + c;
        xs[k] = xk - (double)q * h[k];
    }
    reinterpret_cast<T4*>(b.xs)[i] = mk4((T)xs[0], (T)xs[1], (T)xs[2], (T)0);
}

// ------------------------------------------------------------------------------------
// Half kick + drift.  mode 0 (setup): mirror and noise sums only.
// ------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kTile) k_kick_drift(Bufs b, int mode) {
    using T4 = typename V4<T>::t;
    const TileAtom ta = tile_of(b, blockIdx.x);
    const DevSys& S = b.sys[ta.sys];
    DevState& st = b.st[ta.sys];
    T xs_sum[3] = {(T)0, (T)0, (T)0};
    if ((int)threadIdx.x < ta.count) {
        const int i = ta.first + threadIdx.x;
        const size_t N = b.ntot;
        double xv[3] = {b.x[i], b.x[N + i], b.x[2 * N + i]};
        if (mode == 1) {
            double vv[3] = {b.v[i], b.v[N + i], b.v[2 * N + i]};
            const T4 F = reinterpret_cast<const T4*>(b.F)[i];
            const double c = 0.5 * b.dt / S.mass_e;
            vv[0] += c * (double)F.x; vv[1] += c * (double)F.y; vv[2] += c * (double)F.z;
            for (int k = 0; k < 3; ++k) xv[k] = st.s[k] * xv[k] + (b.dt * st.phi[k]) * vv[k];
            for (int k = 0; k < 3; ++k) { b.v[k * N + i] = vv[k]; b.x[k * N + i] = xv[k]; }
        }
        const int4 q = b.q[i];
        const double m0 = xv[0] - (double)q.x * st.h[0];
        const double m1 = xv[1] - (double)q.y * st.h[1];
        const double m2 = xv[2] - (double)q.z * st.h[2];
        const T4 m = mk4((T)m0, (T)m1, (T)m2, (T)0);
        reinterpret_cast<T4*>(b.xs)[i] = m;
        const T4 mb = reinterpret_cast<const T4*>(b.xsb)[i];
        const T r0 = (T)(st.h[0] / st.hb[0]), r1 = (T)(st.h[1] / st.hb[1]), r2 = (T)(st.h[2] / st.hb[2]);
        const T d0 = m.x - mb.x * r0, d1 = m.y - mb.y * r1, d2 = m.z - mb.z * r2;
        if ((double)(d0 * d0 + d1 * d1 + d2 * d2) > st.thr2 && !st.rebuild) atomicOr(&st.rebuild, 1);
        if (S.tdamp > 0.0) {
            T z[3];
            Noise<T>::xi3(S.seed, (uint64_t)S.rng_id, (uint64_t)st.k, (uint64_t)(i - S.off), z);
            xs_sum[0] = z[0]; xs_sum[1] = z[1]; xs_sum[2] = z[2];
        }
    }
    block_sum_to_acc<T, 3>(xs_sum, b.acc + (size_t)ta.sys * ACC_N * kSlots, ACC_XI, &st.err);
}

// ------------------------------------------------------------------------------------
// Stillinger-Weber force kernel: L lanes per atom, 128/L atoms per block.
// ------------------------------------------------------------------------------------
__device__ __forceinline__ unsigned lanemask_lt() {
    return (1u << (threadIdx.x & 31)) - 1u;
}

template <typename T>
__device__ __forceinline__ void sw_edge(const SWc<T>& P, T r, T& phi, T& dphi, T& g, T& dg) {
    const T s = r * P.inv_sig;
    const T id = (T)1 / (s - P.a);
    const T e1 = exp(id);
    g = exp(P.gam * id);
    T rp, rq;
    if (P.int_pq) {
        const T is2 = (T)1 / (s * s);
        rp = is2 * is2;
        rq = (T)1;
    } else {
        rp = pow(s, -P.p);
        rq = pow(s, -P.q);
    }
    const T poly = P.B * rp - rq;
    phi = P.epsA * poly * e1;
    dphi = P.epsA * e1 * ((-P.p * P.B * rp + P.q * rq) / s - poly * id * id) * P.inv_sig;
    dg = -g * P.gam * id * id * P.inv_sig;
}

template <typename T, int L, int MODE>
__global__ void __launch_bounds__(kTile) k_force(Bufs b) {
    using T4 = typename V4<T>::t;
    constexpr int G = kTile / L;
    __shared__ T4 sh_d[G][kShell];
    __shared__ T sh_g[G][kShell];
    __shared__ T sh_dg[G][kShell];
    __shared__ int sh_e[G][kShell];

    const int tile = blockIdx.x / L, part = blockIdx.x % L;
    const TileAtom ta = tile_of(b, tile);
    const DevSys& S = b.sys[ta.sys];
    DevState& st = b.st[ta.sys];
    const SWc<T> P = reinterpret_cast<const SWc<T>*>(b.swc)[S.prm];
    const int lane = threadIdx.x % L, grp = threadIdx.x / L;
    const unsigned gmask = (L == 32) ? 0xffffffffu : (((1u << L) - 1u) << (((threadIdx.x & 31) / L) * L));
    const T hx = (T)st.h[0], hy = (T)st.h[1], hz = (T)st.h[2];
    const int ia = part * G + grp;
    const bool valid = ia < ta.count;
    const int i = ta.first + ia;
    // per-system mean of this step's thermostat noise (sum of the 32 slots, once per block)
    __shared__ T s_xm[3];
    if (MODE != FM_FORCES && threadIdx.x < 3) {
        const long long* acc = b.acc + (size_t)ta.sys * ACC_N * kSlots + (size_t)(ACC_XI + threadIdx.x) * kSlots;
        long long sum = 0;
        for (int sl = 0; sl < kSlots; ++sl) sum += acc[sl];
        s_xm[threadIdx.x] = (T)((double)sum / kFix / (double)S.n);
    }
    __syncthreads();

    T fx = 0, fy = 0, fz = 0, en = 0;
    T w0 = 0, w1 = 0, w2 = 0, w3 = 0, w4 = 0, w5 = 0;
    bool shell_ovf = false;
    if (valid && S.pot == POT_SW) {
        const T4 xi = reinterpret_cast<const T4*>(b.xs)[i];
        const int ci = min(b.cnt[i], b.cap);
        const int* row = b.nbr + (size_t)i * b.cap;
        int m = 0;
        // phase 1: in-cutoff shell of i, pair terms
        for (int base = 0; base < ci; base += L) {
            const int sidx = base + lane;
            bool in = false;
            T dx = 0, dy = 0, dz = 0, r2 = 0;
            int e = 0;
            if (sidx < ci) {
                e = row[sidx];
                const int j = e & (int)kIndexMask;
                const int code = (int)((unsigned)e >> kCodeShift);
                const T4 xj = reinterpret_cast<const T4*>(b.xs)[j];
                dx = xj.x - xi.x + (T)(code % 3 - 1) * hx;
                dy = xj.y - xi.y + (T)((code / 3) % 3 - 1) * hy;
                dz = xj.z - xi.z + (T)(code / 9 - 1) * hz;
                r2 = dx * dx + dy * dy + dz * dz;
                in = r2 < P.rc2;
            }
            const unsigned bal = __ballot_sync(gmask, in);
            if (in) {
                const int pos = m + __popc(bal & lanemask_lt());
                if (pos < kShell) {
                    const T r = sqrt(r2);
                    T phi, dphi, g, dg;
                    sw_edge<T>(P, r, phi, dphi, g, dg);
                    sh_d[grp][pos] = mk4(dx, dy, dz, r);
                    sh_g[grp][pos] = g;
                    sh_dg[grp][pos] = dg;
                    sh_e[grp][pos] = e;
                    const T c = dphi / r;
                    fx += c * dx; fy += c * dy; fz += c * dz;
                    en += (T)0.5 * phi;
                    const T hc = (T)-0.5 * c;
                    w0 += hc * dx * dx; w1 += hc * dy * dy; w2 += hc * dz * dz;
                    w3 += hc * dx * dy; w4 += hc * dx * dz; w5 += hc * dy * dz;
                }
            }
            m += __popc(bal);
        }
        if (m > kShell) { shell_ovf = true; m = kShell; }
        __syncwarp(gmask);
        // phase 2: triplets centred at i, pairs (a < b) of the shell, flat index dealt mod L
        int t0 = 0;
        for (int a = 0; a < m - 1; ++a) {
            const int rowlen = m - 1 - a;
            int off = (lane - t0) % L;
            if (off < 0) off += L;
            if (off < rowlen) {
                const T4 da = sh_d[grp][a];
                const T ga = sh_g[grp][a], dga = sh_dg[grp][a];
                const T ira = (T)1 / da.w;
                const T uax = da.x * ira, uay = da.y * ira, uaz = da.z * ira;
                for (int bb = a + 1 + off; bb < m; bb += L) {
                    const T4 db = sh_d[grp][bb];
                    const T gb = sh_g[grp][bb], dgb = sh_dg[grp][bb];
                    const T irb = (T)1 / db.w;
                    const T ubx = db.x * irb, uby = db.y * irb, ubz = db.z * irb;
                    const T c = uax * ubx + uay * uby + uaz * ubz;
                    const T dc = c - P.c0;
                    const T two = (T)2 * P.epslam * dc * ga * gb;
                    const T dc2 = P.epslam * dc * dc;
                    // f_a = -dh/dx_a, f_b = -dh/dx_b
                    const T ta_ = two * ira, tb_ = two * irb;
                    const T fax = -(ta_ * (ubx - c * uax) + dc2 * dga * gb * uax);
                    const T fay = -(ta_ * (uby - c * uay) + dc2 * dga * gb * uay);
                    const T faz = -(ta_ * (ubz - c * uaz) + dc2 * dga * gb * uaz);
                    const T fbx = -(tb_ * (uax - c * ubx) + dc2 * ga * dgb * ubx);
                    const T fby = -(tb_ * (uay - c * uby) + dc2 * ga * dgb * uby);
                    const T fbz = -(tb_ * (uaz - c * ubz) + dc2 * ga * dgb * ubz);
                    fx -= fax + fbx; fy -= fay + fby; fz -= faz + fbz;
                    en += dc2 * ga * gb;
                    w0 += da.x * fax + db.x * fbx;
                    w1 += da.y * fay + db.y * fby;
                    w2 += da.z * faz + db.z * fbz;
                    w3 += (T)0.5 * (da.x * fay + da.y * fax + db.x * fby + db.y * fbx);
                    w4 += (T)0.5 * (da.x * faz + da.z * fax + db.x * fbz + db.z * fbx);
                    w5 += (T)0.5 * (da.y * faz + da.z * fay + db.y * fbz + db.z * fby);
                }
            }
            t0 += rowlen;
        }
        // phase 3: triplets centred at each shell neighbour j in which i is a leg
        for (int a = 0; a < m; ++a) {
            const int ea = sh_e[grp][a];
            const int j = ea & (int)kIndexMask;
            const T4 da = sh_d[grp][a];
            const T ga = sh_g[grp][a], dga = sh_dg[grp][a];
            const T rji = da.w, irji = (T)1 / rji;
            const T ux = -da.x * irji, uy = -da.y * irji, uz = -da.z * irji;   // unit j -> i
            const T4 xj = reinterpret_cast<const T4*>(b.xs)[j];
            const int cj = min(b.cnt[j], b.cap);
            const int* rowj = b.nbr + (size_t)j * b.cap;
            for (int sidx = lane; sidx < cj; sidx += L) {
                const int e = rowj[sidx];
                const int k = e & (int)kIndexMask;
                if (k == i) continue;
                const int code = (int)((unsigned)e >> kCodeShift);
                const T4 xk = reinterpret_cast<const T4*>(b.xs)[k];
                const T dx = xk.x - xj.x + (T)(code % 3 - 1) * hx;
                const T dy = xk.y - xj.y + (T)((code / 3) % 3 - 1) * hy;
                const T dz = xk.z - xj.z + (T)(code / 9 - 1) * hz;
                const T r2 = dx * dx + dy * dy + dz * dz;
                if (!(r2 < P.rc2)) continue;
                const T rk = sqrt(r2), irk = (T)1 / rk;
                const T gk = exp(P.gam / (rk * P.inv_sig - P.a));
                const T vx = dx * irk, vy = dy * irk, vz = dz * irk;
                const T c = ux * vx + uy * vy + uz * vz;
                const T dc = c - P.c0;
                const T two = (T)2 * P.epslam * dc * ga * gk * irji;
                const T dc2 = P.epslam * dc * dc * dga * gk;
                fx -= two * (vx - c * ux) + dc2 * ux;
                fy -= two * (vy - c * uy) + dc2 * uy;
                fz -= two * (vz - c * uz) + dc2 * uz;
            }
        }
        // group reduction
#pragma unroll
        for (int o = L / 2; o > 0; o >>= 1) {
            fx += __shfl_xor_sync(gmask, fx, o);
            fy += __shfl_xor_sync(gmask, fy, o);
            fz += __shfl_xor_sync(gmask, fz, o);
            en += __shfl_xor_sync(gmask, en, o);
            w0 += __shfl_xor_sync(gmask, w0, o);
            w1 += __shfl_xor_sync(gmask, w1, o);
            w2 += __shfl_xor_sync(gmask, w2, o);
            w3 += __shfl_xor_sync(gmask, w3, o);
            w4 += __shfl_xor_sync(gmask, w4, o);
            w5 += __shfl_xor_sync(gmask, w5, o);
        }
    }
    if (shell_ovf && lane == 0) atomicOr(&st.err, NEFE_ERR_SHELL_OVERFLOW);

    T red[14];
#pragma unroll
    for (int k = 0; k < 14; ++k) red[k] = (T)0;
    if (valid && lane == 0) {
        const size_t N = b.ntot;
        T fint[3] = {fx, fy, fz};
        T u_int = en, u_ref = 0;
        T fe[3] = {(T)0, (T)0, (T)0};
        if (MODE == FM_FORCES) {
            b.f_out[i] = (double)fint[0]; b.f_out[N + i] = (double)fint[1]; b.f_out[2 * N + i] = (double)fint[2];
            if (b.e_atom) b.e_atom[i] = (double)u_int;
        } else {
            if (S.pot == POT_EINSTEIN || S.k_E > 0.0) {
                // spring displacement from FP64 positions; energies in FP64
                double d[3];
                for (int k = 0; k < 3; ++k) d[k] = b.x[k * N + i] - b.r0[k * N + i];
                const double d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                if (S.pot == POT_EINSTEIN) {
                    u_int = (T)(0.5 * S.k_int * d2);
                    for (int k = 0; k < 3; ++k) fint[k] = (T)(-S.k_int) * (T)d[k];
                }
                if (S.k_E > 0.0) {
                    u_ref = (T)(0.5 * S.k_E * d2);
                    for (int k = 0; k < 3; ++k) fe[k] = (T)(-S.k_E) * (T)d[k];
                }
            }
            double v[3] = {b.v[i], b.v[N + i], b.v[2 * N + i]};
            const T si = (T)st.scale_int, se = (T)st.scale_E;
            T F[3];
            for (int k = 0; k < 3; ++k) F[k] = si * fint[k] + se * fe[k];
            if (S.tdamp > 0.0) {
                T z[3];
                Noise<T>::xi3(S.seed, (uint64_t)S.rng_id, (uint64_t)st.k, (uint64_t)(i - S.off), z);
                const T amp = (T)S.amp, gam = (T)S.gam;
                for (int k = 0; k < 3; ++k) F[k] += -gam * (T)v[k] + amp * (z[k] - s_xm[k]);
            }
            if (MODE == FM_STEP) {
                for (int k = 0; k < 3; ++k) { v[k] += S.ckick * (double)F[k]; b.v[k * N + i] = v[k]; }
            }
            reinterpret_cast<T4*>(b.F)[i] = mk4(F[0], F[1], F[2], (T)0);
            const T me = (T)S.mass_e;
            const T vx = (T)v[0], vy = (T)v[1], vz = (T)v[2];
            red[8] = me * vx * vx;
            red[9] = me * vy * vy;
            red[10] = me * vz * vz;
            red[11] = me * vx * vy;
            red[12] = me * vx * vz;
            red[13] = me * vy * vz;
        }
        red[0] = u_int;
        red[1] = u_ref;
        red[2] = w0; red[3] = w1; red[4] = w2;
        red[5] = w3; red[6] = w4; red[7] = w5;
    }
    block_sum_to_acc<T, 14>(red, b.acc + (size_t)ta.sys * ACC_N * kSlots, ACC_UINT, &st.err);
}

// ------------------------------------------------------------------------------------
// Per-group update (one 128-thread block per system or dCCI pair).
// ------------------------------------------------------------------------------------
__device__ double sched_lambda(const DevSys& S, long long k) {
    double tau = (double)k / (double)S.nsched;
    if (tau > 1.0) tau = 1.0;
    if (S.direction < 0) tau = 1.0 - tau;
    switch (S.sched) {
        case SCHED_FL: {
            const double t2 = tau * tau, t4 = t2 * t2;
            return t4 * tau * (70.0 * t4 - 315.0 * t2 * tau + 540.0 * t2 - 420.0 * tau + 126.0);
        }
        case SCHED_RS: return 1.0 / (1.0 + tau * (1.0 / S.lam_f - 1.0));
        case SCHED_AS: return S.p0 + (S.p1 - S.p0) * tau;
        default: return S.lam0;
    }
}

__device__ void force_scales(const DevSys& S, double lam, double& s_int, double& s_e) {
    if (S.sched == SCHED_FL) { s_int = 1.0 - lam; s_e = lam; }
    else if (S.sched == SCHED_RS || S.pair >= 0) { s_int = lam; s_e = 0.0; }
    else if (S.sched == SCHED_NONE) { s_int = S.lam0; s_e = 0.0; }
    else { s_int = 1.0; s_e = 0.0; }
}

__device__ double target_pressure(const DevSys& S, const DevState& st) {
    if (S.sched == SCHED_RS) return st.lam * S.p_phys;
    if (S.sched == SCHED_AS) return st.lam;
    if (S.pair >= 0) return st.p_tgt;
    return S.p_ext;
}

__device__ void observe(const DevSys& S, DevState& st) {
    const double V = st.box[0] * st.box[1] * st.box[2];
    const double K = 0.5 * (st.kt[0] + st.kt[1] + st.kt[2]);
    for (int k = 0; k < 6; ++k) st.P[k] = (st.kt[k] + st.scale_int * st.vir[k]) / V;
    const double P = (st.P[0] + st.P[1] + st.P[2]) / 3.0;
    double dhdl = 0.0, H;
    if (S.sched == SCHED_FL) {
        dhdl = st.u_ref - st.u_int;
        H = K + (1.0 - st.lam) * st.u_int + st.lam * st.u_ref;
    } else if (S.sched == SCHED_RS) {
        dhdl = st.u_int + S.p_phys * V;
        H = K + st.lam * st.u_int + st.lam * S.p_phys * V;
    } else if (S.sched == SCHED_AS) {
        dhdl = V;
        H = K + st.u_int + st.lam * V;
    } else {
        H = K + st.scale_int * st.u_int + (S.baro != BARO_NONE ? target_pressure(S, st) * V : 0.0);
    }
    st.V = V;
    st.dHdl = dhdl;
    st.H = H;
    (void)P;
}

__device__ void record_and_kick(const DevSys& S, DevState& st, double dt, double* trace) {
    const double P = (st.P[0] + st.P[1] + st.P[2]) / 3.0;
    st.sums[0] += st.H; st.sums[1] += st.dHdl; st.sums[2] += P; st.sums[3] += st.V; st.sums[4] += 1.0;
    if (S.trace_every > 0 && S.trace_cap > 0 && st.k % S.trace_every == 0) {
        double* r = trace + (S.trace_off + st.trace_n % S.trace_cap) * 9;
        r[0] = (double)st.k; r[1] = st.lam; r[2] = st.W; r[3] = st.dHdl; r[4] = st.u_int;
        r[5] = st.V; r[6] = P * kEvA3ToGPa; r[7] = target_pressure(S, st) * kEvA3ToGPa;
        r[8] = (st.kt[0] + st.kt[1] + st.kt[2]) / ((3.0 * S.n - 3.0) * kB);
        st.trace_n += 1;
    }
    if (S.baro != BARO_NONE) {
        const double Qb = (S.n + 1) * kB * S.T * S.pdamp * S.pdamp;
        const double ptgt = target_pressure(S, st);
        if (S.baro == BARO_ISO) {
            const double g = 3.0 * st.V * (P - ptgt) / Qb;
            for (int k = 0; k < 3; ++k) st.eta[k] += dt * g;
        } else {
            for (int k = 0; k < 3; ++k) st.eta[k] += dt * st.V * (st.P[k] - ptgt) / Qb;
        }
    }
}

__device__ void prepare_step(const DevSys& S, DevState& st, double dt) {
    force_scales(S, st.lam, st.scale_int, st.scale_E);
    double maxrel = 0.0;
    for (int k = 0; k < 3; ++k) {
        const double z = st.eta[k] * dt;
        st.s[k] = exp(z);
        st.phi[k] = (z != 0.0) ? expm1(z) / z : 1.0;
        st.box[k] *= st.s[k];
        st.h[k] = st.box[k] / (double)st.ncell[k];
        maxrel = fmax(maxrel, fabs(st.h[k] / st.hb[k] - 1.0));
    }
    const double thr = 0.5 * (S.skin - maxrel * S.rcs);
    st.thr2 = thr > 0.0 ? thr * thr : -1.0;
}

__global__ void __launch_bounds__(kTile) k_group(Bufs b, const DevGroup* groups, int mode) {
    const DevGroup gr = groups[blockIdx.x];
    const int members[2] = {gr.a, gr.b};
    const int nm = gr.b >= 0 ? 2 : 1;
    // decode the slot sums (fixed order: deterministic)
    if (mode != 0) {
        for (int mi = 0; mi < nm; ++mi) {
            const int s = members[mi];
            DevState& st = b.st[s];
            const long long* acc = b.acc + (size_t)s * ACC_N * kSlots;
            if (threadIdx.x < ACC_N && threadIdx.x < ACC_XI) {
                long long sum = 0;
                for (int sl = 0; sl < kSlots; ++sl) sum += acc[(size_t)threadIdx.x * kSlots + sl];
                const double v = (double)sum / kFix;
                const int a = threadIdx.x;
                if (a == ACC_UINT) st.u_int = v;
                else if (a == ACC_UREF) st.u_ref = v;
                else if (a < ACC_KT) st.vir[a - ACC_VIR] = v;
                else st.kt[a - ACC_KT] = v;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        for (int mi = 0; mi < nm; ++mi) {
            const int s = members[mi];
            if (mode == 0) {
                const DevSys& S = b.sys[s];
                DevState& st = b.st[s];
                if (S.pair >= 0) {
                    const DevPair& pr = b.pairs[S.pair];
                    st.lam = 1.0;
                    st.p_tgt = pr.ps;
                } else if (S.sched != SCHED_NONE) {
                    st.lam = sched_lambda(S, st.k);
                }
                force_scales(S, st.lam, st.scale_int, st.scale_E);
                for (int k = 0; k < 3; ++k) { st.s[k] = 1.0; st.phi[k] = 1.0; }
            } else {
                observe(b.sys[s], b.st[s]);
            }
        }
        if (mode == 1) {
            for (int mi = 0; mi < nm; ++mi) {
                const int s = members[mi];
                record_and_kick(b.sys[s], b.st[s], b.dt, b.trace);
            }
            if (gr.pair >= 0) {
                DevPair& pr = b.pairs[gr.pair];
                DevState& A = b.st[gr.a];
                DevState& B = b.st[gr.b];
                const DevSys& SA = b.sys[gr.a];
                const DevSys& SB = b.sys[gr.b];
                const double du = A.u_int / SA.n - B.u_int / SB.n;
                const double dv = A.V / SA.n - B.V / SB.n;
                double lam_next, ps_next;
                const double tau1 = fmin((double)(pr.k + 1) / (double)pr.nsteps, 1.0);
                const double tau0 = fmin((double)pr.k / (double)pr.nsteps, 1.0);
                if (pr.mode == 0) {
                    const double T1 = pr.frm + (pr.to - pr.frm) * tau1;
                    lam_next = pr.frm / T1;
                    if (fabs(dv) < 1e-6) {
                        pr.err |= NEFE_ERR_DEGEN;
                        lam_next = pr.lam; ps_next = pr.ps;
                    } else {
                        ps_next = pr.ps - (lam_next - pr.lam) * (du / dv);
                    }
                } else {
                    const double p0 = pr.frm + (pr.to - pr.frm) * tau0;
                    const double p1 = pr.frm + (pr.to - pr.frm) * tau1;
                    if (fabs(du) < 1e-12) {
                        pr.err |= NEFE_ERR_DEGEN;
                        lam_next = pr.lam; ps_next = pr.ps;
                    } else {
                        lam_next = pr.lam * (1.0 + p0 * dv / du) / (1.0 + p1 * dv / du);
                        ps_next = lam_next * p1;
                    }
                }
                pr.lam = lam_next;
                pr.ps = ps_next;
                pr.k += 1;
                A.lam = B.lam = lam_next;
                A.p_tgt = B.p_tgt = ps_next;
                if (pr.err) { atomicOr(&A.err, pr.err); atomicOr(&B.err, pr.err); }
            } else {
                const DevSys& S = b.sys[gr.a];
                DevState& st = b.st[gr.a];
                if (S.sched != SCHED_NONE) {
                    const double lam_next = sched_lambda(S, st.k + 1);
                    st.W += st.dHdl * (lam_next - st.lam);
                    st.lam = lam_next;
                }
            }
            for (int mi = 0; mi < nm; ++mi) {
                const int s = members[mi];
                DevState& st = b.st[s];
                prepare_step(b.sys[s], st, b.dt);
                st.rebuild = 0;
                st.k += 1;
            }
        }
    }
    if (mode != 2) {
        __syncthreads();
        for (int mi = 0; mi < nm; ++mi) {
            long long* acc = b.acc + (size_t)members[mi] * ACC_N * kSlots;
            for (int t = threadIdx.x; t < ACC_N * kSlots; t += blockDim.x) acc[t] = 0;
        }
    }
}

__global__ void k_noise(unsigned long long seed, unsigned long long sys, unsigned long long step, int n,
                        int prec, double* xi) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (prec == NEFE_FP64) {
        double z[3];
        Noise<double>::xi3(seed, sys, step, (uint64_t)i, z);
        for (int k = 0; k < 3; ++k) xi[3 * i + k] = z[k];
    } else {
        float z[3];
        Noise<float>::xi3(seed, sys, step, (uint64_t)i, z);
        for (int k = 0; k < 3; ++k) xi[3 * i + k] = (double)z[k];
    }
}

// ------------------------------------------------------------------------------------
// Launchers
// ------------------------------------------------------------------------------------
bool lanes_supported(int lanes) { return lanes == 4 || lanes == 8 || lanes == 16 || lanes == 32; }

void launch_cells(const Bufs& b, int precision, int ntiles, int nsys, int force_all,
                  cudaStream_t s, long* launches) {
    if (ntiles <= 0) return;
    if (precision == NEFE_FP64) k_cells_count<double><<<ntiles, kTile, 0, s>>>(b, force_all);
    else k_cells_count<float><<<ntiles, kTile, 0, s>>>(b, force_all);
    k_cells_scan<<<nsys, 256, 0, s>>>(b, force_all);
    k_cells_fill<<<ntiles, kTile, 0, s>>>(b, force_all);
    k_cells_sort<<<nsys, 256, 0, s>>>(b, force_all);
    if (launches) *launches += 4;
}

void launch_cells_and_list(const Bufs& b, int precision, int ntiles, int nsys, int force_all,
                           cudaStream_t s, long* launches) {
    if (ntiles <= 0) return;
    launch_cells(b, precision, ntiles, nsys, force_all, s, launches);
    if (precision == NEFE_FP64) k_nlist<double><<<ntiles, kTile, 0, s>>>(b, force_all);
    else k_nlist<float><<<ntiles, kTile, 0, s>>>(b, force_all);
    if (launches) *launches += 1;
}

// (n,3) row-major <-> SoA with stride n.
__global__ void k_aos_to_soa(const double* __restrict__ a, double* __restrict__ s, int n) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 3 * n) return;
    const int i = t / 3, k = t % 3;
    s[(size_t)k * n + i] = a[t];
}
__global__ void k_soa_to_aos(const double* __restrict__ s, double* __restrict__ a, int n) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 3 * n) return;
    const int i = t / 3, k = t % 3;
    a[t] = s[(size_t)k * n + i];
}
void launch_aos_soa(const double* src, double* dst, int n, int to_soa, cudaStream_t s) {
    if (n <= 0) return;
    const int blocks = (3 * n + 255) / 256;
    if (to_soa) k_aos_to_soa<<<blocks, 256, 0, s>>>(src, dst, n);
    else k_soa_to_aos<<<blocks, 256, 0, s>>>(src, dst, n);
}

__global__ void k_decode_ev(const long long* acc, double* out7) {
    const int t = threadIdx.x;
    if (t >= 7) return;
    const int a = t == 0 ? ACC_UINT : ACC_VIR + (t - 1);
    long long sum = 0;
    for (int sl = 0; sl < kSlots; ++sl) sum += acc[(size_t)a * kSlots + sl];
    out7[t] = (double)sum / kFix;
}

void launch_decode_ev(const long long* acc, double* out7, cudaStream_t s) {
    k_decode_ev<<<1, 32, 0, s>>>(acc, out7);
}

void launch_kick_drift(const Bufs& b, int precision, int ntiles, int mode, cudaStream_t s, long* launches) {
    if (ntiles <= 0) return;
    if (precision == NEFE_FP64) k_kick_drift<double><<<ntiles, kTile, 0, s>>>(b, mode);
    else k_kick_drift<float><<<ntiles, kTile, 0, s>>>(b, mode);
    if (launches) *launches += 1;
}

void launch_mirror(const Bufs& b, int precision, int ntiles, cudaStream_t s, long* launches) {
    if (ntiles <= 0) return;
    if (precision == NEFE_FP64) k_mirror<double><<<ntiles, kTile, 0, s>>>(b);
    else k_mirror<float><<<ntiles, kTile, 0, s>>>(b);
    if (launches) *launches += 1;
}

template <typename T, int MODE>
static void force_dispatch(const Bufs& b, int lanes, int ntiles, cudaStream_t s) {
    switch (lanes) {
        case 4:
            // the FP64 shell of 32 groups does not fit the 48 KB static shared limit
            if (sizeof(T) == 8) k_force<T, 8, MODE><<<ntiles * 8, kTile, 0, s>>>(b);
            else k_force<float, 4, MODE><<<ntiles * 4, kTile, 0, s>>>(b);
            break;
        case 8: k_force<T, 8, MODE><<<ntiles * 8, kTile, 0, s>>>(b); break;
        case 16: k_force<T, 16, MODE><<<ntiles * 16, kTile, 0, s>>>(b); break;
        default: k_force<T, 32, MODE><<<ntiles * 32, kTile, 0, s>>>(b); break;
    }
}

void launch_force(const Bufs& b, int precision, int lanes, int ntiles, int mode, cudaStream_t s,
                  long* launches) {
    if (ntiles <= 0) return;
    if (precision == NEFE_FP64) {
        if (mode == FM_FORCES) force_dispatch<double, FM_FORCES>(b, lanes, ntiles, s);
        else if (mode == FM_SETUP) force_dispatch<double, FM_SETUP>(b, lanes, ntiles, s);
        else force_dispatch<double, FM_STEP>(b, lanes, ntiles, s);
    } else {
        if (mode == FM_FORCES) force_dispatch<float, FM_FORCES>(b, lanes, ntiles, s);
        else if (mode == FM_SETUP) force_dispatch<float, FM_SETUP>(b, lanes, ntiles, s);
        else force_dispatch<float, FM_STEP>(b, lanes, ntiles, s);
    }
    if (launches) *launches += 1;
}

void launch_group(const Bufs& b, const DevGroup* groups, int ngroups, int mode, cudaStream_t s,
                  long* launches) {
    if (ngroups <= 0) return;
    k_group<<<ngroups, kTile, 0, s>>>(b, groups, mode);
    if (launches) *launches += 1;
}

void launch_noise(unsigned long long seed, unsigned long long sys_id, unsigned long long step, int n,
                  int precision, double* xi, cudaStream_t s) {
    if (n <= 0) return;
    k_noise<<<(n + 127) / 128, 128, 0, s>>>(seed, sys_id, step, n, precision, xi);
}

}  // namespace nefe
