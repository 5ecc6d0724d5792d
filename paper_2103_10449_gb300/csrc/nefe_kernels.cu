// libnefe device kernels for sm_103a.
//
// Step sequence of one time step k -> k+1 (all systems of a context at once):
//   k_group       per system / dCCI pair: reads the fixed-point sums of step k, observes
//                 P, V, dH/dl, records, kicks the barostat, advances lambda and W (Eq. Wdyn,
//                 left point), applies the dCCI update (Eqs. Ps_coex_discreted /
//                 l_coex_discreted), sets this step's drift factors and zeroes the sums.
//   k_kick_drift  v += dt/2 F/m; displacement since the last list build += dt phi v (+ the
//                 affine box drift), kept as a compensated pair in the FP32 path; mirror
//                 xs = x - q h; displacement test -> rebuild flag; thermostat noise + its sum.
//                 In the scatter form this work is done by the previous step's epilogue for the
//                 systems without a barostat (k_finish with fuse), and the kernel skips them.
//   rebuild       (flagged systems) fold the displacement into the FP64 anchor, cell count ->
//                 scan -> fill (with a cell-ordered copy of the mirror) -> Verlet list; as a
//                 kernel sequence, or as one cooperative launch (k_rebuild_coop).
//   k_edges1      force pass A, one thread per atom: in-cutoff shell of each atom, pair terms,
//                 the shell's moments and the force the triplets centred on the atom exert on
//                 each leg atom; in the scatter form (the FP32 default) every leg force and the
//                 atom's own force go into int32 fixed-point accumulators (order independent).
//                 k_edges: the lane-group variants (and the FP64 path), storing per edge.
//   k_finish      the scatter form's epilogue: reads and clears the accumulators; Einstein
//                 springs, lambda mixing, Langevin force with its per-system mean removed,
//                 second half kick (and the next step's kick, drift and noise, see above).
//   k_gather      force pass B of the gather form: the atom's pass-A force plus the leg forces
//                 that the triplets centred on its neighbours exert on it, then the same
//                 epilogue.
//
// Positions: the FP64 anchor x (positions at the last list build) plus the displacement
// since then (FP64, or an FP32 value + FP32 compensation term, ~2^-48 relative).  The anchor
// absorbs the displacement at every list build, so the per-step path of the FP32 kernels
// issues no FP64 instruction (GB300 runs FP64 at 1/64 of the FP32 rate): per-system
// constants are read from FP32 copies written once per step by k_group.
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

// Precision-explicit math (no silent promotion of FP32 arguments to the FP64 routines).
// The FP32 path uses the hardware approximations (MUFU: ex2, rcp, rsqrt; a few ulp, far
// inside the 1e-5 relative force tolerance); the FP64 path the correctly rounded routines.
__device__ __forceinline__ float xexp(float v) { return __expf(v); }
__device__ __forceinline__ double xexp(double v) { return ::exp(v); }
__device__ __forceinline__ float xrcp(float v) { return __fdividef(1.0f, v); }
__device__ __forceinline__ double xrcp(double v) { return 1.0 / v; }
__device__ __forceinline__ float xrsqrt(float v) { return rsqrtf(v); }
__device__ __forceinline__ double xrsqrt(double v) { return ::rsqrt(v); }
__device__ __forceinline__ float xpow(float a, float b) { return __powf(a, b); }
__device__ __forceinline__ float xlog(float v) { return __logf(v); }
__device__ __forceinline__ double xlog(double v) { return ::log(v); }
__device__ __forceinline__ double xpow(double a, double b) { return ::pow(a, b); }

// FP32 copy or FP64 source of a constant, by kernel precision.
template <typename T> __device__ __forceinline__ T pick(double d, float f) {
    if constexpr (sizeof(T) == 4) return f; else return d;
}

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
        const double r0 = ::sqrt(-2.0 * ::log(u0)), r1 = ::sqrt(-2.0 * ::log(u2));
        double s0, c0, s1, c1;
        ::sincos(two_pi * u1, &s0, &c0);
        ::sincos(two_pi * u3, &s1, &c1);
        out[0] = r0 * c0; out[1] = r0 * s0; out[2] = r1 * c1;
    }
};
template <> struct Noise<float> {
    __device__ static void xi3(uint64_t seed, uint64_t sys, uint64_t step, uint64_t id, float out[3]) {
        uint64_t c[4] = {step, id, sys, 0ULL};
        philox4x64_10(c, seed, 0ULL);
        const float u0 = ((float)(uint32_t)(c[0] >> 40) + 0.5f) * 0x1p-24f;
        const float u1 = ((float)(uint32_t)(c[1] >> 40) + 0.5f) * 0x1p-24f;
        const float u2 = ((float)(uint32_t)(c[2] >> 40) + 0.5f) * 0x1p-24f;
        const float u3 = ((float)(uint32_t)(c[3] >> 40) + 0.5f) * 0x1p-24f;
        const float r0 = sqrtf(-2.0f * logf(u0)), r1 = sqrtf(-2.0f * logf(u2));
        float s0, c0, s1, c1;
        sincospif(2.0f * u1, &s0, &c0);
        sincospif(2.0f * u3, &s1, &c1);
        out[0] = r0 * c0; out[1] = r0 * s0; out[2] = r1 * c1;
    }
};

// ------------------------------------------------------------------------------------
// Deterministic per-system sums: warp shuffle in kernel precision, then the block's warp
// partials summed in kernel precision in a fixed order, then one int64 fixed-point atomic per
// value into slot (blockIdx % kSlots).  The FP64 path converts the block sum at 2^-32; the
// FP32 path rounds it to a multiple of 2^-16 (an int32 conversion, |block sum| < 32768) before
// moving it to the 2^-32 scale, so a block's contribution carries at most 2^-17 of rounding
// on top of its FP32 summation error.  Integer addition makes the per-system total independent
// of the order in which blocks arrive.  Every thread of the block must call it.
// ------------------------------------------------------------------------------------
template <typename T, int K>
__device__ __forceinline__ void block_sum_to_acc(T (&v)[K], long long* acc_sys, int first,
                                                 unsigned* err) {
    __shared__ T red[kTile / 32][K];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        T x = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) red[w][k] = x;
    }
    __syncthreads();
    if (threadIdx.x < K) {
        T s = 0;
        const int nw = (int)(blockDim.x >> 5);
        for (int i = 0; i < nw; ++i) s += red[i][threadIdx.x];
        long long q;
        bool bad;
        if constexpr (sizeof(T) == 4) {
            // round(s 2^16) in int32 (|s| < 32768 per block), moved to the 2^-32 scale
            const float t = s * 65536.0f;
            bad = !(fabsf(t) < 2147483520.0f);
            q = bad ? 0LL : (long long)__float2int_rn(t) * 65536LL;
        } else {
            bad = !isfinite(s);
            q = bad ? 0LL : __double2ll_rn(s * kFix);
        }
        if (bad) {
            atomicOr(err, NEFE_ERR_NAN);
        } else if (q != 0) {
            atomicAdd(reinterpret_cast<unsigned long long*>(
                          &acc_sys[(size_t)(first + threadIdx.x) * kSlots + (blockIdx.x % kSlots)]),
                      (unsigned long long)q);
        }
    }
}

// Sum of the kSlots fixed-point slots of one per-system value.  The loads are independent, so
// they are issued together (one memory latency, not kSlots of them).
__device__ __forceinline__ long long slot_sum(const long long* slots) {
    long long v[kSlots];
#pragma unroll
    for (int sl = 0; sl < kSlots; ++sl) v[sl] = slots[sl];
    long long sum = 0;
#pragma unroll
    for (int sl = 0; sl < kSlots; ++sl) sum += v[sl];
    return sum;
}

// Per-block table of the 27 cell-offset vectors o h (o in {-1,0,1}^3), indexed by the list
// entry's code.  Every thread of the block must call it.
template <typename T>
__device__ __forceinline__ void offset_table(typename V4<T>::t* tab, T hx, T hy, T hz) {
    if (threadIdx.x < 27) {
        const int c = threadIdx.x;
        const int ox = c % 3 - 1, oy = (c / 3) % 3 - 1, oz = c / 9 - 1;
        tab[c] = mk4(ox == 0 ? (T)0 : (ox < 0 ? -hx : hx), oy == 0 ? (T)0 : (oy < 0 ? -hy : hy),
                     oz == 0 ? (T)0 : (oz < 0 ? -hz : hz), (T)0);
    }
    __syncthreads();
}

// The same 27 offset vectors as three component rows of 32 (row k, entry c at tab[32 k + c]):
// a warp whose lanes index different entries reads each row without bank conflicts (a table
// of 16-byte vectors indexed at random serialises).  Every thread of the block must call it.
template <typename T>
__device__ __forceinline__ void offset_rows(T* tab, T hx, T hy, T hz) {
    if (threadIdx.x < 27) {
        const int c = threadIdx.x;
        const int ox = c % 3 - 1, oy = (c / 3) % 3 - 1, oz = c / 9 - 1;
        tab[c] = ox == 0 ? (T)0 : (ox < 0 ? -hx : hx);
        tab[32 + c] = oy == 0 ? (T)0 : (oy < 0 ? -hy : hy);
        tab[64 + c] = oz == 0 ? (T)0 : (oz < 0 ? -hz : hz);
    }
    __syncthreads();
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

// FP32 copies of the box-dependent constants (called wherever h or hb change).
__device__ __forceinline__ void refresh_box_f(DevState& st) {
    bool hm = false;
    for (int k = 0; k < 3; ++k) {
        st.h_f[k] = (float)st.h[k];
        st.hb_f[k] = (float)st.hb[k];
        st.rho_f[k] = (float)(st.h[k] / st.hb[k]);
        hm = hm || (st.h[k] != st.hb[k]);
    }
    st.hmoved = hm ? 1 : 0;
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

// A tile's system descriptor and state copied into shared memory by all threads of the block
// (independent 4-byte loads: one memory latency, instead of one per cache line of the structs
// that the kernel's field accesses would otherwise wait for, one after the other), and the tile.
// Writes to the state (flags, error bits) still go to the global copy.  Every thread of the block
// must call it; it ends with a barrier.
struct StagedSys {
    DevSys S;
    DevState st;
};
__device__ __forceinline__ TileAtom stage_tile(const Bufs& b, int tile, StagedSys& sh) {
    const int sys = b.tile_sys[tile];
    const uint32_t* gs = reinterpret_cast<const uint32_t*>(b.sys + sys);
    const uint32_t* gt = reinterpret_cast<const uint32_t*>(b.st + sys);
    uint32_t* ds = reinterpret_cast<uint32_t*>(&sh.S);
    uint32_t* dt = reinterpret_cast<uint32_t*>(&sh.st);
    constexpr int ws = (int)(sizeof(DevSys) / 4), wt = (int)(sizeof(DevState) / 4);
    for (int w = threadIdx.x; w < ws + wt; w += blockDim.x) {
        if (w < ws) ds[w] = gs[w];
        else dt[w - ws] = gt[w - ws];
    }
    __syncthreads();
    TileAtom t;
    t.sys = sys;
    t.first = sh.S.off + (tile - sh.S.tile0) * kTile;
    t.count = min(kTile, sh.S.off + sh.S.n - t.first);
    return t;
}

// ------------------------------------------------------------------------------------
// Rebuild R1: fold the displacement into the FP64 anchor; cell of each atom, unwrapped cell
// index q, fresh mirror, spring offset, occupancy count.  The cell formula is
// c = (int)(w n) with w = x/L - floor(x/L) evaluated in FP64.
// ------------------------------------------------------------------------------------
template <typename T>
__device__ void cells_count_tile(const Bufs& b, int tile) {
    using T4 = typename V4<T>::t;
    const TileAtom ta = tile_of(b, tile);
    const DevSys& S = b.sys[ta.sys];
    DevState& st = b.st[ta.sys];
    __shared__ int s_n3[3];
    __shared__ double s_h[3], s_ib[3];
    if (b.rtiles) {                              // engine: the grid was set by k_rebuild_list
        if (threadIdx.x < 3) {
            s_n3[threadIdx.x] = st.ncell[threadIdx.x];
            s_h[threadIdx.x] = st.h[threadIdx.x];
            s_ib[threadIdx.x] = st.ibox[threadIdx.x];
        }
    } else if (threadIdx.x == 0) {               // the grid of this tile's system, once per tile
        int g3[3];
        const bool ok = grid_for(st.box, S.rcs, S.ncell_cap, g3);
        for (int k = 0; k < 3; ++k) {
            s_n3[k] = g3[k];
            s_h[k] = __ddiv_rn(st.box[k], (double)g3[k]);
            s_ib[k] = __ddiv_rn(1.0, st.box[k]);
        }
        if (tile == S.tile0) {
            for (int k = 0; k < 3; ++k) { st.ncell[k] = g3[k]; st.h[k] = s_h[k]; st.hb[k] = s_h[k]; }
            refresh_box_f(st);
            st.nbuild += 1;
            if (!ok) atomicOr(&st.err, NEFE_ERR_BOX);
        }
    }
    __syncthreads();
    const int n3[3] = {s_n3[0], s_n3[1], s_n3[2]};
    const double h[3] = {s_h[0], s_h[1], s_h[2]};
    const double ib[3] = {s_ib[0], s_ib[1], s_ib[2]};
    // The stateless cell sort reproduces the plain definition (x / L, correctly rounded); the
    // engine's list build only needs a consistent cell for each atom (its cells are at least
    // rcs (1 + 1e-9) wide and the list decision itself is exact), so it multiplies by 1/L
    // instead of dividing (FP64 division is a long instruction sequence on this GPU).
    const bool exact = b.rtiles == nullptr;
    __syncthreads();                             // the next tile of the loop rewrites the table
    if ((int)threadIdx.x >= ta.count) return;
    const int i = ta.first + threadIdx.x;
    const size_t N = b.ntot;
    int c3[3], qv[3];
    double xm[3], sd[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < 3; ++k) {
        double xk = b.x[k * N + i];
        if (b.dhi) {   // fold the displacement into the FP64 anchor
            T* dh = reinterpret_cast<T*>(b.dhi);
            T* dl = reinterpret_cast<T*>(b.dlo);
            const double d = (double)dh[k * N + i] + (b.dlo ? (double)dl[k * N + i] : 0.0);
            xk = xk + d;
            b.x[k * N + i] = xk;
            dh[k * N + i] = (T)0;
            if (b.dlo) dl[k * N + i] = (T)0;
        }
        const double s = exact ? __ddiv_rn(xk, st.box[k]) : xk * ib[k];
        const double fl = floor(s);
        const double w = __dsub_rn(s, fl);
        int c = (int)__dmul_rn(w, (double)n3[k]);
        if (c >= n3[k]) c = n3[k] - 1;
        if (c < 0) c = 0;
        c3[k] = c;
        qv[k] = (int)fl * n3[k] + c;
        xm[k] = xk - (double)qv[k] * h[k];
        if (b.r0) sd[k] = xk - b.r0[k * N + i];
    }
    const int cell = c3[0] + n3[0] * (c3[1] + n3[1] * c3[2]);
    b.cell_of[i] = cell;
    b.q[i] = make_int4(qv[0], qv[1], qv[2], 0);
    const T4 m = mk4((T)xm[0], (T)xm[1], (T)xm[2], (T)0);
    reinterpret_cast<T4*>(b.xs)[i] = m;
    if (b.xa) reinterpret_cast<T4*>(b.xa)[i] = m;
    if (b.sd0) reinterpret_cast<T4*>(b.sd0)[i] = mk4((T)sd[0], (T)sd[1], (T)sd[2], (T)0);
    atomicAdd(&b.cell_count[S.cell0 + cell], 1);
}

// The rebuild kernels walk a worklist of the tiles of flagged systems (written by
// k_rebuild_list) with a bounded grid, or every tile (stateless calls: no worklist).
#define NEFE_FOR_TILES(b, body_call)                                           \
    do {                                                                      \
        if ((b).rtiles) {                                                     \
            const int n_ = *(b).rcount;                                       \
            for (int w_ = blockIdx.x; w_ < n_; w_ += gridDim.x) {             \
                const int tile = (b).rtiles[w_];                              \
                body_call;                                                    \
            }                                                                 \
        } else {                                                              \
            const int tile = blockIdx.x;                                      \
            body_call;                                                        \
        }                                                                     \
    } while (0)

template <typename T>
__global__ void __launch_bounds__(kTile) k_cells_count(Bufs b) {
    NEFE_FOR_TILES(b, cells_count_tile<T>(b, tile));
}

// Worklist of the tiles of every system whose rebuild flag is set (all with force_all), and the
// cell grid of each such system at its current box (per axis floor(L/rcs) reduced while
// L/n < rcs (1 + 1e-9), h = L/n, 1/L), computed once per system here rather than per tile, and
// only when the box or the list radius differ from the ones the grid was last computed for
// (the FP64 divisions are skipped for every system at fixed volume).
// Tile order in the list does not matter: every tile is processed independently.
// With b.rebuild_all, a step on which any system's flag is set rebuilds every system (the flags
// of all are set here, so the later rebuild kernels see them): rebuilding a list early never
// changes what the force passes compute, and one build over the whole batch runs its kernels at
// full width where many small builds, one per step, each pay their latency.
// The worklist of one step, built by one block (any multiple of 32 threads up to 256).
__device__ void build_worklist(const Bufs& b, int nsys, int force_all) {
    __shared__ int cnt;
    // no flag set anywhere this step (b.any_rebuild[0], written wherever a flag is): empty worklist
    if (!force_all && b.any_rebuild && *(volatile int*)b.any_rebuild == 0) {
        if (threadIdx.x == 0) {
            *b.rcount = 0;
            if (b.rcbase) b.rcbase[nsys] = 0;
        }
        return;
    }
    if (threadIdx.x == 0) cnt = 0;
    if (b.rebuild_all && !force_all) {
        int any = 0;
        for (int s = threadIdx.x; s < nsys; s += blockDim.x) any |= b.st[s].rebuild;
        if (__syncthreads_or(any))
            for (int s = threadIdx.x; s < nsys; s += blockDim.x) b.st[s].rebuild = 1;
    }
    __syncthreads();
    for (int s = threadIdx.x; s < nsys; s += blockDim.x) {
        DevState& st = b.st[s];
        if (force_all || st.rebuild) {
            const DevSys& S = b.sys[s];
            const int base = atomicAdd(&cnt, S.ntile);
            for (int t = 0; t < S.ntile; ++t) b.rtiles[base + t] = S.tile0 + t;
            const double bx[3] = {st.box[0], st.box[1], st.box[2]};
            const bool same = st.grcs == S.rcs && st.gbox[0] == bx[0] && st.gbox[1] == bx[1] &&
                              st.gbox[2] == bx[2];
            if (!same) {
                int g3[3];
                const bool ok = grid_for(bx, S.rcs, S.ncell_cap, g3);
                for (int k = 0; k < 3; ++k) {
                    st.ncell[k] = g3[k];
                    st.h[k] = __ddiv_rn(bx[k], (double)g3[k]);
                    st.hb[k] = st.h[k];
                    st.ibox[k] = __ddiv_rn(1.0, bx[k]);
                    st.gbox[k] = bx[k];
                }
                st.grcs = S.rcs;
                refresh_box_f(st);
                if (!ok) atomicOr(&st.err, NEFE_ERR_BOX);
            }
            st.nbuild += 1;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) *b.rcount = cnt;
    if (b.rcbase) {   // first worklist cell of each system: exclusive scan of the flagged cell counts
        __shared__ int wsum[8];
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
        int carry = 0;
        for (int base = 0; base < nsys; base += (int)blockDim.x) {
            const int s = base + (int)threadIdx.x;
            int v = 0;
            if (s < nsys) {
                const DevState& st = b.st[s];
                if (force_all || st.rebuild) v = st.ncell[0] * st.ncell[1] * st.ncell[2];
            }
            int incl = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            if (lane == 31) wsum[w] = incl;
            __syncthreads();
            int woff = 0, tot = 0;
            for (int k = 0; k < nw; ++k) {
                if (k < w) woff += wsum[k];
                tot += wsum[k];
            }
            if (s < nsys) b.rcbase[s] = carry + woff + incl - v;
            carry += tot;
            __syncthreads();
        }
        if (threadIdx.x == 0) b.rcbase[nsys] = carry;
    }
}

__global__ void __launch_bounds__(256) k_rebuild_list(Bufs b, int nsys, int force_all) {
    build_worklist(b, nsys, force_all);
}

// R2: exclusive scan of system s's cell occupancy by one block (blockDim a multiple of 32, at
// most 256; 8 consecutive cells per thread per pass); resets the counts.
__device__ void scan_system_cells(const Bufs& b, int s) {
    constexpr int PT = 8;
    const DevSys& S = b.sys[s];
    DevState& st = b.st[s];
    const int ncells = st.ncell[0] * st.ncell[1] * st.ncell[2];
    int* start = b.cell_start + S.cell0 + s;
    int* count = b.cell_count + S.cell0;
    int* cursor = b.cell_cursor + S.cell0;
    __shared__ int warp_tot[8];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
    const int span = (int)blockDim.x * PT;
    int carry = 0;
    for (int base = 0; base < ncells; base += span) {
        const int c0 = base + (int)threadIdx.x * PT;
        int v[PT], tsum = 0;
#pragma unroll
        for (int u = 0; u < PT; ++u) {
            v[u] = c0 + u < ncells ? count[c0 + u] : 0;
            tsum += v[u];
        }
        int incl = tsum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) warp_tot[w] = incl;
        __syncthreads();
        int woff = 0, tot = 0;
        for (int k = 0; k < nw; ++k) {
            if (k < w) woff += warp_tot[k];
            tot += warp_tot[k];
        }
        int run = carry + woff + incl - tsum;
#pragma unroll
        for (int u = 0; u < PT; ++u) {
            if (c0 + u < ncells) {
                start[c0 + u] = run;
                cursor[c0 + u] = run;
                count[c0 + u] = 0;
            }
            run += v[u];
        }
        carry += tot;
        __syncthreads();                         // warp_tot is rewritten by the next pass
    }
    if (threadIdx.x == 0) {
        start[ncells] = carry;
        if (carry != S.n) atomicOr(&st.err, NEFE_ERR_CELL);
    }
}

// One 256-thread block per system; systems whose rebuild flag is clear return (all are scanned
// with force_all).
__global__ void __launch_bounds__(256) k_cells_scan(Bufs b, int force_all) {
    const int s = blockIdx.x;
    if (!force_all && !b.st[s].rebuild) return;
    scan_system_cells(b, s);
}

// Atom index carried in the .w lane of a position vector (bit pattern in FP32, value in FP64).
template <typename T> __device__ __forceinline__ T pack_index(int i);
template <> __device__ __forceinline__ float pack_index<float>(int i) { return __int_as_float(i); }
template <> __device__ __forceinline__ double pack_index<double>(int i) { return (double)i; }
__device__ __forceinline__ int unpack_index(float w) { return __float_as_int(w); }
__device__ __forceinline__ int unpack_index(double w) { return (int)w; }

// R3: scatter atoms into their cell segment (order inside a cell fixed by R4), with a copy
// of their mirror positions in the same order for the list build.
template <typename T>
__device__ void cells_fill_tile(const Bufs& b, int tile) {
    using T4 = typename V4<T>::t;
    const TileAtom ta = tile_of(b, tile);
    const DevSys& S = b.sys[ta.sys];
    if ((int)threadIdx.x >= ta.count) return;
    const int i = ta.first + threadIdx.x;
    const int pos = atomicAdd(&b.cell_cursor[S.cell0 + b.cell_of[i]], 1);
    if (pos < 0 || pos >= S.n) {                 // inconsistent occupancy: record, never write out of range
        atomicOr(&b.st[ta.sys].err, NEFE_ERR_CELL);
        return;
    }
    b.perm[S.off + pos] = i;
    if (b.xcs) {
        const T4 m = reinterpret_cast<const T4*>(b.xs)[i];
        reinterpret_cast<T4*>(b.xcs)[S.off + pos] = mk4(m.x, m.y, m.z, pack_index<T>(i));
    }
}
template <typename T>
__global__ void __launch_bounds__(kTile) k_cells_fill(Bufs b) {
    NEFE_FOR_TILES(b, cells_fill_tile<T>(b, tile));
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
        const int lo = max(0, min(start[c], S.n)), hi = max(lo, min(start[c + 1], S.n));
        for (int a = lo + 1; a < hi; ++a) {
            const int key = p[a];
            int z = a - 1;
            while (z >= lo && p[z] > key) { p[z + 1] = p[z]; --z; }
            p[z + 1] = key;
        }
    }
}

// Index of entry k of atom i's Verlet row (see Bufs::nbr_il).  The interleaved form lets the
// lanes of a warp that take consecutive atoms read their next four entries as one contiguous
// 512-byte request.
__device__ __forceinline__ size_t nbr_at(const Bufs& b, int i, int k) {
    return b.nbr_il ? ((size_t)(k >> 2) * b.ntot + i) * 4 + (k & 3) : (size_t)i * b.cap + k;
}

// Padding of an interleaved row past its mrow entries up to the next multiple of 4: atom i's
// own image through cell offset (-1, -1, -1), at distance |(h_x, h_y, h_z)| >= sqrt(3) rcs
// from i, so it never enters a shell (the force passes read whole groups of four).
__device__ __forceinline__ void pad_row(const Bufs& b, int i, int mrow, int lane, int nlanes) {
    if (!b.nbr_il) return;
    const int end = (mrow + 3) & ~3;
    for (int k = mrow + lane; k < end && k < b.cap; k += nlanes) b.nbr[nbr_at(b, i, k)] = i;
}

// Debug build (NEFE_DEBUG_BOUNDS, libnefe_debug.so): every atom index read from device data
// (list entries, shell entries, UF rows) is checked before it is used; an index outside the
// context's atoms sets NEFE_ERR_CELL in the system's error word and the access is skipped (a
// list entry is replaced by the row's padding entry, which never enters a shell).  In the
// normal build the check compiles away.
#ifdef NEFE_DEBUG_BOUNDS
#define NEFE_IN_RANGE(idx, n, errp) \
    (((unsigned)(idx) < (unsigned)(n)) ? true : (atomicOr((errp), (unsigned)NEFE_ERR_CELL), false))
#else
#define NEFE_IN_RANGE(idx, n, errp) true
#endif

// Exact list criterion in FP64, the plain definition: raw = x_j - x_i, m = rint(raw/L),
// d = raw - m L, ((d_x^2 + d_y^2) + d_z^2) < rcs^2; every operation rounded separately.
__device__ __noinline__ bool exact_pair_in(const Bufs& b, const double box[3], int i, int j,
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

// R5: Verlet list, L lanes per atom (a group of L lanes of one warp).
// The 27 neighbour cells of atom i's cell form 9 x-rows (one per (oy, oz)); the three cells of
// a row (ox = -1, 0, 1) are consecutive in the cell-ordered mirror copy unless the row wraps at
// the box edge (cx = 0 or cx = nx - 1), so a row is one contiguous range of candidates (two
// pieces where it wraps).  A cell whose box is farther than rcs from atom i is pruned, which
// trims a row at its ends or drops it.  The pieces are concatenated into one candidate sequence
// of the group, which its lanes walk L at a time (lane l takes candidates l, l + L, ...: every
// lane but the last pass's is busy); the cell offset of a candidate follows from its position
// against its piece's cell boundaries.  A candidate is accepted or rejected on its mirror
// distance when that lies outside a relative band of 1e-4 (FP32) / 1e-10 (FP64) around rcs^2,
// and inside the band by the exact FP64 criterion (which must also agree with the offset's
// image), so the list equals the plain definition bit for bit.  Accepted entries are appended
// through a ballot, as keys j * 32 + o, and then ranked by atom index into the row, which
// fixes the order.
constexpr int kRebuildBlocks = 152 * 8;   // bounded grid of the worklist-driven rebuild kernels
constexpr int kRowPieces = 18;            // piece p of row r at 2 r + p
constexpr int kKeyRow = kMaxCap + 4;      // key buffer row: 16-byte aligned, groups on different banks

// Per-group tables of the list build in shared memory.
template <typename T>
struct NlistShared {
    using T4 = typename V4<T>::t;
    int4 pc[kRowPieces];          // (first candidate in xcs, start of its 2nd cell, of its 3rd cell, first flat index)
    T4 ps[kRowPieces];            // (x_i - ox h_x, y_i - oy h_y, z_i - oz h_z) of the piece's first cell
    int code[kRowPieces];         // cell-offset code of the piece's first cell
    int flat_end;                 // number of candidates of the group
};

// One piece of row (oy, oz): cells x0 .. x0 + nc - 1 of the row starting at rb (consecutive in
// memory), as (first candidate, end, start of the second cell, start of the third cell), the
// last two INT_MAX when absent.
__device__ __forceinline__ int4 row_piece(const int* start, int rb, int x0, int nc, int n) {
    const int lo = max(0, min(start[rb + x0], n));
    const int hi = max(lo, min(start[rb + x0 + nc], n));
    const int b1 = nc > 1 ? start[rb + x0 + 1] : INT_MAX;
    const int b2 = nc > 2 ? start[rb + x0 + 2] : INT_MAX;
    return make_int4(lo, hi, b1, b2);
}

template <typename T, int L>
__device__ void nlist_item(const Bufs& b, int tile, int part, unsigned (*keys)[kKeyRow],
                           NlistShared<T>* tab) {
    using T4 = typename V4<T>::t;
    constexpr int G = kTile / L;
    constexpr int RR = (9 + L - 1) / L;          // rows per lane
    const TileAtom ta = tile_of(b, tile);
    const DevSys& S = b.sys[ta.sys];
    if (S.pot != POT_SW) {                       // no SW term: no SW list (uniform over the block)
        const int ia = part * G + (int)threadIdx.x / L;
        if (threadIdx.x % L == 0 && ia < ta.count) b.cnt[ta.first + ia] = 0;
        return;
    }
    DevState& st = b.st[ta.sys];
    const int lane = threadIdx.x % L, grp = threadIdx.x / L;
    const int lbase = ((threadIdx.x & 31) / L) * L;
    NlistShared<T>& sh = tab[grp];
    const int ia = part * G + grp;
    // groups past the tile's end stay in the warp-uniform loops below with no candidates
    const bool valid = ia < ta.count;
    const int i = ta.first + (valid ? ia : 0);
    const int nx = st.ncell[0], ny = st.ncell[1], nz = st.ncell[2];
    const int cell = b.cell_of[i];
    const int cx = cell % nx, cy = (cell / nx) % ny, cz = cell / (nx * ny);
    const int* start = b.cell_start + S.cell0 + ta.sys;
    const T4 xi = reinterpret_cast<const T4*>(b.xs)[i];
    const T hx = pick<T>(st.h[0], st.h_f[0]), hy = pick<T>(st.h[1], st.h_f[1]), hz = pick<T>(st.h[2], st.h_f[2]);
    T lo2, hi2;
    if constexpr (sizeof(T) == 4) {
        lo2 = S.rcs2_lo_f;
        hi2 = S.rcs2_hi_f;
    } else {
        lo2 = S.rcs * S.rcs * (1.0 - 1e-10);
        hi2 = S.rcs * S.rcs * (1.0 + 1e-10);
    }
    // pruning bound: relaxed by 1e-3 of rcs^2, far above the rounding of the mirror positions
    // (which lie in [0, h) of their own cell), so no pair within rcs can be missed
    const T prune2 = (T)(S.rcs * S.rcs * 1.001);
    const T4* xc = reinterpret_cast<const T4*>(b.xcs) + S.off;
    // first ox of a row's second piece: the row wraps between ox = -1 and 0 (cx = 0) or between
    // 0 and +1 (cx = nx - 1); 2 when it does not wrap (nx >= 2, so never both)
    const int brk = cx == 0 ? 0 : (cx == nx - 1 ? 1 : 2);
    int carry = 0;
#pragma unroll
    for (int k = 0; k < RR; ++k) {
        const int r = lane + k * L;
        int4 p0 = make_int4(0, 0, INT_MAX, INT_MAX), p1 = p0;
        int a = 0, a2 = 0, cb = 0;
        if (valid && r < 9) {
            const int oy = r % 3 - 1, oz = r / 3 - 1;
            const T ey = oy < 0 ? xi.y : (oy > 0 ? hy - xi.y : (T)0);
            const T ez = oz < 0 ? xi.z : (oz > 0 ? hz - xi.z : (T)0);
            const T fy = ey > (T)0 ? ey : (T)0, fz = ez > (T)0 ? ez : (T)0;
            const T fyz = fy * fy + fz * fz;
            cb = 3 * (oy + 1) + 9 * (oz + 1);
            if (fyz <= prune2) {
                const T fl = xi.x > (T)0 ? xi.x : (T)0, fr = hx - xi.x > (T)0 ? hx - xi.x : (T)0;
                a = fl * fl + fyz <= prune2 ? -1 : 0;          // lower cell kept
                const int e = fr * fr + fyz <= prune2 ? 1 : 0; // upper cell kept
                int yy = cy + oy, zz = cz + oz;
                yy = yy < 0 ? yy + ny : (yy >= ny ? yy - ny : yy);
                zz = zz < 0 ? zz + nz : (zz >= nz ? zz - nz : zz);
                const int rb = nx * (yy + ny * zz);
                const int e1 = min(e, brk - 1);               // first piece: ox = a .. e1
                if (a <= e1) {
                    int x0 = cx + a;
                    x0 = x0 < 0 ? x0 + nx : x0;
                    p0 = row_piece(start, rb, x0, e1 - a + 1, S.n);
                }
                a2 = max(a, brk);                             // second piece: ox = a2 .. e
                if (brk < 2 && a2 <= e) {
                    int x0 = cx + a2;
                    x0 = x0 >= nx ? x0 - nx : x0;
                    p1 = row_piece(start, rb, x0, e - a2 + 1, S.n);
                }
            }
            const T yo = xi.y - (T)oy * hy, zo = xi.z - (T)oz * hz;
            sh.ps[2 * r] = mk4(xi.x - (T)a * hx, yo, zo, (T)0);
            sh.ps[2 * r + 1] = mk4(xi.x - (T)a2 * hx, yo, zo, (T)0);
            sh.code[2 * r] = cb + a + 1;
            sh.code[2 * r + 1] = cb + a2 + 1;
        }
        // flat positions: exclusive scan of the rows' lengths over the group, row order
        const int n0 = p0.y - p0.x, len = n0 + (p1.y - p1.x);
        int incl = len;
#pragma unroll
        for (int o = 1; o < L; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o, L);
            if (lane >= o) incl += y;
        }
        const int f0 = carry + incl - len;
        if (valid && r < 9) {
            sh.pc[2 * r] = make_int4(p0.x, p0.z, p0.w, f0);
            sh.pc[2 * r + 1] = make_int4(p1.x, p1.z, p1.w, f0 + n0);
        }
        carry += __shfl_sync(0xffffffffu, incl, L - 1, L);
    }
    if (lane == 0) sh.flat_end = carry;
    __syncwarp();
    // walk the flat sequence L candidates at a time; the pass count is uniform over the warp
    const int total = carry;
    const int npass = __reduce_max_sync(0xffffffffu, (total + L - 1) / L);
    int cnt = 0;
    for (int pass = 0; pass < npass; ++pass) {
        const int t = pass * L + lane;
        bool in = false, band = false, bad = false;
        unsigned key = 0u;
        T dx = (T)0, dy = (T)0, dz = (T)0;
        int j = 0;
        if (t < total) {                         // straight-line: no branch inside
            int e = 0;                           // piece of t: last entry whose flat start is <= t
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                const int c = e + step;
                if (c < kRowPieces && sh.pc[c].w <= t) e = c;
            }
            const int4 pc = sh.pc[e];
            const T4 po = sh.ps[e];
            const int p = pc.x + (t - pc.w);
            const T4 xj = xc[p];
            j = unpack_index(xj.w);
            const int inc = (p >= pc.y ? 1 : 0) + (p >= pc.z ? 1 : 0);
            const int o = sh.code[e] + inc;
            dx = (xj.x - po.x) + (T)inc * hx;
            dy = xj.y - po.y;
            dz = xj.z - po.z;
            const T dd = dx * dx + dy * dy + dz * dz;
            bad = (unsigned)(j - S.off) >= (unsigned)S.n;
            const bool cand = !bad && !(j == i && o == 13);
            in = cand && dd < lo2;
            band = cand && !(dd < lo2) && dd <= hi2;
            key = (unsigned)j * 32u + (unsigned)o;
        }
        if (__any_sync(0xffffffffu, bad || band)) {   // rare: a corrupt cell table or the exact test
            if (bad) atomicOr(&st.err, NEFE_ERR_CELL);
            if (band) {
                double d[3];
                in = exact_pair_in(b, st.box, i, j, __dmul_rn(S.rcs, S.rcs), d);
                in = in && fabs(d[0] - (double)dx) < 0.5 * st.h[0] &&
                     fabs(d[1] - (double)dy) < 0.5 * st.h[1] &&
                     fabs(d[2] - (double)dz) < 0.5 * st.h[2];
            }
        }
        const unsigned bal = __ballot_sync(0xffffffffu, in);
        const unsigned m = (L == 32) ? bal : ((bal >> lbase) & ((1u << L) - 1u));
        const int pos = cnt + __popc(m & ((1u << lane) - 1u));
        if (in && pos < kMaxCap) keys[grp][pos] = key;
        cnt += __popc(m);
    }
    // rank by atom index into the row (indices in a row are distinct); the key row is padded to
    // a multiple of 4 with the largest key, so it is read 4 keys at a time
    const int have = cnt < kMaxCap ? cnt : kMaxCap;
    const int have4 = (have + 3) & ~3;
    for (int z = have + lane; z < have4; z += L) keys[grp][z] = 0xffffffffu;
    __syncwarp();
    if (valid) {
        const int cap = b.cap;
        const int mrow = cnt < cap ? cnt : cap;
        const uint4* row4 = reinterpret_cast<const uint4*>(keys[grp]);
        constexpr int R = 4;
        for (int a0 = 0; a0 < have; a0 += R * L) {
            unsigned k[R];
            int rk[R];
#pragma unroll
            for (int u = 0; u < R; ++u) {
                const int a = a0 + u * L + lane;
                k[u] = a < have ? keys[grp][a] : 0xffffffffu;
                rk[u] = 0;
            }
            for (int z = 0; z < have4; z += 4) {
                const uint4 v = row4[z >> 2];
#pragma unroll
                for (int u = 0; u < R; ++u)
                    rk[u] += (v.x < k[u] ? 1 : 0) + (v.y < k[u] ? 1 : 0) + (v.z < k[u] ? 1 : 0) +
                             (v.w < k[u] ? 1 : 0);
            }
#pragma unroll
            for (int u = 0; u < R; ++u) {
                const int a = a0 + u * L + lane;
                if (a < have && rk[u] < mrow)
                    b.nbr[nbr_at(b, i, rk[u])] = (int)((k[u] >> 5) | ((k[u] & 31u) << kCodeShift));
            }
        }
        pad_row(b, i, mrow, lane, L);
        if (lane == 0) {
            b.cnt[i] = cnt;
            if (cnt > cap) atomicOr(&st.err, NEFE_ERR_NBR_OVERFLOW);
        }
    }
    __syncwarp();                                // shared tables reused by the next item
}

template <typename T, int L>
__global__ void __launch_bounds__(kTile, 8) k_nlist(Bufs b) {
    constexpr int G = kTile / L;
    __shared__ __align__(16) unsigned keys[G][kKeyRow];
    __shared__ NlistShared<T> tab[G];
    if (b.rtiles) {
        const int n = *b.rcount * L;
        for (int w = blockIdx.x; w < n; w += gridDim.x) nlist_item<T, L>(b, b.rtiles[w / L], w % L, keys, tab);
    } else {
        nlist_item<T, L>(b, blockIdx.x / L, blockIdx.x % L, keys, tab);
    }
}

// R5 (list mode 0, the default): one warp per cell.  The atoms of a cell share its 27 neighbour
// cells, so the warp walks that candidate sequence once (its 9 x-rows as pieces, 32 candidates
// at a time, one per lane: position, image offset and index loaded once) and tests every
// candidate against each atom of the cell in turn (the cell's atoms up to 8 at a time, their
// positions in shared memory), with the same filter, band and exact test as above.  An accepted
// key j * 32 + o is appended to the cell atom's shared row through a shared-memory counter (in
// whatever order the lanes arrive), and the rows are then ranked by key, i.e. by atom index,
// one key per lane, which fixes the order.  Every candidate position is read once per
// neighbouring cell instead of once per neighbouring atom.
constexpr int kHomeChunk = 8;             // cell atoms per walk of the candidate sequence
template <typename T>
struct CellListShared {
    using T4 = typename V4<T>::t;
    unsigned keys[kHomeChunk][kKeyRow];   // accepted keys of each cell atom
    T4 home[kHomeChunk];                  // cell atoms: mirror position, index in .w
    int4 pc[kRowPieces];                  // (first candidate, start of 2nd cell, of 3rd cell, first flat index)
    T4 po[kRowPieces];                    // offset (ox h_x, oy h_y, oz h_z) of the piece's first cell
    int code[kRowPieces];                 // cell-offset code of the piece's first cell
    int pw[kRowPieces];                   // first flat index of each piece (the .w of pc again, as
                                          // one int row: the search reads it without conflicts)
    int cnt[kHomeChunk];                  // accepted count of each cell atom (append cursor)
    unsigned sorted[kKeyRow];             // the row being written, in rank order
};

template <typename T>
__device__ __forceinline__ void nlist_cell(const Bufs& b, int s, int c, CellListShared<T>& sh, int lane) {
    using T4 = typename V4<T>::t;
    constexpr unsigned kAll = 0xffffffffu;
    const DevSys& S = b.sys[s];
    DevState& st = b.st[s];
    const int* start = b.cell_start + S.cell0 + s;
    const int n = S.n, off = S.off;
    const int hs = max(0, min(start[c], n)), he = max(hs, min(start[c + 1], n));
    const int m = he - hs;
    if (m == 0) return;
    const T4* xc = reinterpret_cast<const T4*>(b.xcs) + off;
    if (S.pot != POT_SW) {                       // no SW term: no SW list
        for (int q = lane; q < m; q += 32) {
            const int i = unpack_index(xc[hs + q].w);
            if ((unsigned)(i - off) < (unsigned)n) b.cnt[i] = 0;
        }
        return;
    }
    const int nx = st.ncell[0], ny = st.ncell[1], nz = st.ncell[2];
    const int cx = c % nx, cy = (c / nx) % ny, cz = c / (nx * ny);
    const T hx = pick<T>(st.h[0], st.h_f[0]), hy = pick<T>(st.h[1], st.h_f[1]), hz = pick<T>(st.h[2], st.h_f[2]);
    T lo2, hi2;
    if constexpr (sizeof(T) == 4) {
        lo2 = S.rcs2_lo_f;
        hi2 = S.rcs2_hi_f;
    } else {
        lo2 = S.rcs * S.rcs * (1.0 - 1e-10);
        hi2 = S.rcs * S.rcs * (1.0 + 1e-10);
    }
    // the rows: lane r < 9 builds row r = (oy, oz) as one piece (ox = -1 .. 1), or two where it
    // wraps at the box edge (cx = 0: the piece ox = -1, then 0 .. 1; cx = nx - 1: -1 .. 0, then 1)
    const int brk = cx == 0 ? 0 : (cx == nx - 1 ? 1 : 2);
    int len = 0, n0 = 0;
    int4 p0 = make_int4(0, 0, INT_MAX, INT_MAX), p1 = p0;
    int a2 = 0;
    if (lane < 9) {
        const int oy = lane % 3 - 1, oz = lane / 3 - 1;
        int yy = cy + oy, zz = cz + oz;
        yy = yy < 0 ? yy + ny : (yy >= ny ? yy - ny : yy);
        zz = zz < 0 ? zz + nz : (zz >= nz ? zz - nz : zz);
        const int rb = nx * (yy + ny * zz);
        const int e1 = min(1, brk - 1);
        a2 = brk;
        if (-1 <= e1) p0 = row_piece(start, rb, cx == 0 ? nx - 1 : cx - 1, e1 + 2, n);
        if (brk < 2) p1 = row_piece(start, rb, cx + a2 >= nx ? cx + a2 - nx : cx + a2, 2 - a2, n);
        n0 = p0.y - p0.x;
        len = n0 + (p1.y - p1.x);
    }
    int incl = len;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kAll, incl, o);
        if (lane >= o) incl += y;
    }
    const int total = __shfl_sync(kAll, incl, 31);
    if (lane < 9) {
        const int oy = lane % 3 - 1, oz = lane / 3 - 1;
        const int f0 = incl - len;
        const T offy = (T)oy * hy, offz = (T)oz * hz;
        const int cb = 3 * (oy + 1) + 9 * (oz + 1);
        sh.pw[2 * lane] = f0;
        sh.pw[2 * lane + 1] = f0 + n0;
        sh.pc[2 * lane] = make_int4(p0.x, p0.z, p0.w, f0);
        sh.po[2 * lane] = mk4(-hx, offy, offz, (T)0);
        sh.code[2 * lane] = cb;
        sh.pc[2 * lane + 1] = make_int4(p1.x, p1.z, p1.w, f0 + n0);
        sh.po[2 * lane + 1] = mk4((T)a2 * hx, offy, offz, (T)0);
        sh.code[2 * lane + 1] = cb + a2 + 1;
    }
    __syncwarp();
    const int cap = b.cap;
    for (int h0 = 0; h0 < m; h0 += kHomeChunk) {
        const int mh = min(kHomeChunk, m - h0);
        if (lane < mh) sh.home[lane] = xc[hs + h0 + lane];
        if (lane < kHomeChunk) sh.cnt[lane] = 0;
        __syncwarp();
        for (int t0 = 0; t0 < total; t0 += 32) {
            const int t = t0 + lane;
            int j = -1, o = 0;
            // a candidate that is not one (past the sequence, or a bad index) sits far away, so
            // the distance test below rejects it without a separate flag
            T cxj = (T)1e30, cyj = (T)1e30, czj = (T)1e30;
            if (t < total) {
                int e = 0;                       // piece of t: last entry whose flat start is <= t
#pragma unroll
                for (int step = 16; step > 0; step >>= 1) {
                    const int q = e + step;
                    if (q < kRowPieces && sh.pw[q] <= t) e = q;
                }
                const int4 pc = sh.pc[e];
                const T4 po = sh.po[e];
                const int p = pc.x + (t - pc.w);
                const T4 xj = xc[p];
                j = unpack_index(xj.w);
                const int inc = (p >= pc.y ? 1 : 0) + (p >= pc.z ? 1 : 0);
                o = sh.code[e] + inc;
                if ((unsigned)(j - off) < (unsigned)n) {
                    cxj = xj.x + (po.x + (T)inc * hx);
                    cyj = xj.y + po.y;
                    czj = xj.z + po.z;
                } else {
                    atomicOr(&st.err, NEFE_ERR_CELL);
                }
            }
            // The common path is the distance test alone; the few candidates inside the upper
            // edge of the band (about one in six) are then checked for being the atom itself,
            // and decided by the exact FP64 criterion when they fall inside the band.  Each
            // accepted key is appended through a shared-memory counter: the order of the keys in
            // a row buffer does not matter, since the row is ranked by key below.
            for (int a = 0; a < mh; ++a) {
                const T4 ha = sh.home[a];
                const T dx = cxj - ha.x, dy = cyj - ha.y, dz = czj - ha.z;
                const T dd = dx * dx + dy * dy + dz * dz;
                if (dd <= hi2) {
                    const int ia = unpack_index(ha.w);
                    bool in = !(j == ia && o == 13);
                    if (in && !(dd < lo2)) {     // rare: decided by the exact FP64 criterion
                        double d[3];
                        in = exact_pair_in(b, st.box, ia, j, __dmul_rn(S.rcs, S.rcs), d);
                        in = in && fabs(d[0] - (double)dx) < 0.5 * st.h[0] &&
                             fabs(d[1] - (double)dy) < 0.5 * st.h[1] &&
                             fabs(d[2] - (double)dz) < 0.5 * st.h[2];
                    }
                    if (in) {
                        const int pos = atomicAdd(&sh.cnt[a], 1);
                        if (pos < kMaxCap) sh.keys[a][pos] = (unsigned)j * 32u + (unsigned)o;
                    }
                }
            }
        }
        __syncwarp();
        const int cnt = lane < kHomeChunk ? sh.cnt[lane] : 0;   // lane a: accepted count of cell atom a
        // rank each cell atom's keys by atom index (one key per lane; the row padded to a
        // multiple of 4 with the largest key and read 4 keys at a time)
        for (int a = 0; a < mh; ++a) {
            const int ca = __shfl_sync(kAll, cnt, a);
            const int ia = unpack_index(sh.home[a].w);
            const int have = ca < kMaxCap ? ca : kMaxCap;
            const int have4 = (have + 3) & ~3;
            if (have + lane < have4) sh.keys[a][have + lane] = 0xffffffffu;
            __syncwarp();
            const int mrow = ca < cap ? ca : cap;
            const uint4* row4 = reinterpret_cast<const uint4*>(sh.keys[a]);
            for (int k0 = 0; k0 < have; k0 += 32) {
                const int kk = k0 + lane;
                const unsigned key = kk < have ? sh.keys[a][kk] : 0xffffffffu;
                int rk = 0;
                for (int z = 0; z < have4; z += 4) {
                    const uint4 v = row4[z >> 2];
                    rk += (v.x < key ? 1 : 0) + (v.y < key ? 1 : 0) + (v.z < key ? 1 : 0) + (v.w < key ? 1 : 0);
                }
                if (kk < have && rk < mrow) sh.sorted[rk] = key;
            }
            __syncwarp();
            // the row in rank order, four entries per lane and store (one 16-byte vector of an
            // interleaved row, padded past mrow; consecutive lanes write consecutive entries of
            // a row-major row)
            for (int g = lane; 4 * g < mrow; g += 32) {
                int v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int k = 4 * g + u;
                    const unsigned key = k < mrow ? sh.sorted[k] : 0u;
                    v[u] = k < mrow ? (int)((key >> 5) | ((key & 31u) << kCodeShift)) : ia;
                }
                if (b.nbr_il) {
                    reinterpret_cast<int4*>(b.nbr)[(size_t)g * b.ntot + ia] = make_int4(v[0], v[1], v[2], v[3]);
                } else {
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        if (4 * g + u < mrow) b.nbr[(size_t)ia * cap + 4 * g + u] = v[u];
                }
            }
            if (lane == 0) {
                b.cnt[ia] = ca;
                if (ca > cap) atomicOr(&st.err, NEFE_ERR_NBR_OVERFLOW);
            }
        }
        __syncwarp();                            // the home table and key rows are reused
    }
}

// Each warp takes a contiguous range of the worklist cells: with a worklist, the cells of the
// flagged systems in system order (rcbase[s] = first worklist cell of system s, rcbase[nsys] =
// their number); without one (stateless calls, one system), every cell of system 0.
template <typename T>
__device__ void nlist_cells_of_grid(const Bufs& b, int nsys, CellListShared<T>* shm) {
    const int lane = threadIdx.x & 31;
    CellListShared<T>& sh = shm[threadIdx.x >> 5];
    const int nw = gridDim.x * (kTile / 32);
    const int wid = blockIdx.x * (kTile / 32) + (int)(threadIdx.x >> 5);
    int C;
    if (b.rcbase) {
        C = b.rcbase[nsys];
    } else {
        const DevState& s0 = b.st[0];
        C = s0.ncell[0] * s0.ncell[1] * s0.ncell[2];
    }
    const int K = (C + nw - 1) / nw;
    const int g0 = wid * K, g1 = min(C, g0 + K);
    if (g0 >= g1) return;
    int s = 0;
    if (b.rcbase) {                              // largest s with rcbase[s] <= g0
        int lo = 0, hi = nsys;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (b.rcbase[mid] <= g0) lo = mid; else hi = mid;
        }
        s = lo;
    }
    for (int g = g0; g < g1; ++g) {
        if (b.rcbase) {
            while (s + 1 < nsys && b.rcbase[s + 1] <= g) ++s;
        }
        nlist_cell<T>(b, s, g - (b.rcbase ? b.rcbase[s] : 0), sh, lane);
    }
}

template <typename T>
__global__ void __launch_bounds__(kTile, 8) k_nlist_cell(Bufs b, int nsys) {
    __shared__ CellListShared<T> shm[kTile / 32];
    nlist_cells_of_grid<T>(b, nsys, shm);
}

// ------------------------------------------------------------------------------------
// The engine's whole rebuild in one cooperative launch (all blocks resident): worklist (block
// 0), cell count, scan, fill and list build, separated by grid barriers.  On a step where no list
// is stale every block returns at once, so the step pays one near-empty launch instead of five.
//
// Grid barrier: one 32-bit word; block 0 adds 2^31 - (nblocks - 1), every other block adds 1, so
// the word's top bit flips exactly when the last block arrives and its low bits return to what
// they were (the word needs no reset between barriers or launches).  Each block waits for the
// top bit it saw to flip, for at most kBarrierNs of %globaltimer; a block that gives up sets the
// context's timeout word and NEFE_ERR_TIMEOUT in every system and returns (the host then reports
// NEFE_ETIMEOUT and resets the words).  The launch is cooperative, so the wait never depends on a
// block that is not resident.
// ------------------------------------------------------------------------------------
constexpr unsigned long long kBarrierNs = 1000000000ULL;   // 1 s

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Returns false (in every thread of the block) when the wait gave up.
__device__ bool grid_barrier(unsigned* word, int* timeout, unsigned long long limit_ns, unsigned nblocks) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned add = blockIdx.x == 0 ? 0x80000000u - (nblocks - 1u) : 1u;
        __threadfence();
        const unsigned old = atomicAdd(word, add);
        int ok = 1;
        const unsigned long long t0 = global_ns();
        while (((*(volatile unsigned*)word ^ old) & 0x80000000u) == 0u) {
            if (global_ns() - t0 > limit_ns) {
                ok = 0;
                atomicOr(timeout, 1);
                break;
            }
            __nanosleep(64);
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

__device__ void flag_timeout(const Bufs& b, int nsys) {
    for (int s = threadIdx.x; s < nsys; s += blockDim.x) atomicOr(&b.st[s].err, NEFE_ERR_TIMEOUT);
}

template <typename T>
__global__ void __launch_bounds__(kTile, 8) k_rebuild_coop(Bufs b, int nsys) {
    __shared__ CellListShared<T> shm[kTile / 32];
    // no flag set anywhere this step: the word is written only by the kernels before this one
    if (*(volatile int*)b.any_rebuild == 0) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            *b.rcount = 0;
            b.rcbase[nsys] = 0;
        }
        return;
    }
    unsigned* bar = reinterpret_cast<unsigned*>(b.any_rebuild + 3);
    int* tmo = b.any_rebuild + 2;
    const unsigned nb = gridDim.x;
    if (blockIdx.x == 0) build_worklist(b, nsys, 0);
    if (!grid_barrier(bar, tmo, kBarrierNs, nb)) { flag_timeout(b, nsys); return; }
    NEFE_FOR_TILES(b, cells_count_tile<T>(b, tile));
    if (!grid_barrier(bar, tmo, kBarrierNs, nb)) { flag_timeout(b, nsys); return; }
    for (int sy = blockIdx.x; sy < nsys; sy += gridDim.x)
        if (b.st[sy].rebuild) scan_system_cells(b, sy);
    if (!grid_barrier(bar, tmo, kBarrierNs, nb)) { flag_timeout(b, nsys); return; }
    NEFE_FOR_TILES(b, cells_fill_tile<T>(b, tile));
    if (!grid_barrier(bar, tmo, kBarrierNs, nb)) { flag_timeout(b, nsys); return; }
    nlist_cells_of_grid<T>(b, nsys, shm);
}

// Test of the barrier's time limit: a grid whose barrier expects one block more than it has
// (nothing will ever complete it), with a short limit; every block gives up and sets *timeout.
__global__ void __launch_bounds__(kTile) k_barrier_selftest(unsigned* word, int* timeout, unsigned long long ns) {
    grid_barrier(word, timeout, ns, gridDim.x + 1u);
}

// ------------------------------------------------------------------------------------
// Uhlenbeck-Ford fluid (the liquid's reference system, Sec. 2.1):
//   u(r) = -p kT ln(1 - exp(-r^2/sigma^2)) - u(rc),  r < rc.
// R6 (rebuild): UF pair rows.  One thread per atom walks the 125 cells o in {-2..2}^3 around its
// own (cells are at least rcs wide and rc + skin <= 2 rcs, so they cover the list radius; with
// at least 5 cells per axis no cell is visited twice) and appends every j within the list
// radius (rc + skin, FP32 mirror distance with a relative margin of 1e-5: the list only has
// to contain every pair that can come within rc before the next rebuild).  Rows are in cell
// order, not sorted: the force kernel sums in fixed point, so the order does not matter.
// ------------------------------------------------------------------------------------
template <typename T>
__device__ void uflist_tile(const Bufs& b, int tile) {
    using T4 = typename V4<T>::t;
    const TileAtom ta = tile_of(b, tile);
    const DevSys& S = b.sys[ta.sys];
    if (S.uf_mode == UF_NONE) return;            // uniform over the block
    DevState& st = b.st[ta.sys];
    if ((int)threadIdx.x >= ta.count) return;
    const int i = ta.first + threadIdx.x;
    const int nx = st.ncell[0], ny = st.ncell[1], nz = st.ncell[2];
    if (nx < 5 || ny < 5 || nz < 5) {
        b.uf_cnt[i] = 0;
        atomicOr(&st.err, NEFE_ERR_BOX);
        return;
    }
    const int cell = b.cell_of[i];
    const int cx = cell % nx, cy = (cell / nx) % ny, cz = cell / (nx * ny);
    const int* start = b.cell_start + S.cell0 + ta.sys;
    const T4 xi = reinterpret_cast<const T4*>(b.xs)[i];
    const T hx = pick<T>(st.h[0], st.h_f[0]), hy = pick<T>(st.h[1], st.h_f[1]), hz = pick<T>(st.h[2], st.h_f[2]);
    const T R2 = pick<T>(S.uf_R2 * (1.0 + 1e-5), S.uf_R2_f * (1.0f + 1e-5f));
    const T4* xc = reinterpret_cast<const T4*>(b.xcs) + S.off;
    int* row = b.uf_nbr + (size_t)i * kUfCap;
    int count = 0;
    for (int oz = -2; oz <= 2; ++oz) {
        int zz = cz + oz;
        zz = zz < 0 ? zz + nz : (zz >= nz ? zz - nz : zz);
        for (int oy = -2; oy <= 2; ++oy) {
            int yy = cy + oy;
            yy = yy < 0 ? yy + ny : (yy >= ny ? yy - ny : yy);
            for (int ox = -2; ox <= 2; ++ox) {
                int xx = cx + ox;
                xx = xx < 0 ? xx + nx : (xx >= nx ? xx - nx : xx);
                const int c2 = xx + nx * (yy + ny * zz);
                const int lo = max(0, min(start[c2], S.n)), hi = max(lo, min(start[c2 + 1], S.n));
                const T offx = (T)ox * hx, offy = (T)oy * hy, offz = (T)oz * hz;
                const unsigned code = (unsigned)((ox + 2) + 5 * (oy + 2) + 25 * (oz + 2));
                for (int q = lo; q < hi; ++q) {
                    const T4 xj = xc[q];
                    const int j = unpack_index(xj.w);
                    if (j < S.off || j >= S.off + S.n) {
                        atomicOr(&st.err, NEFE_ERR_CELL);
                        continue;
                    }
                    if (j == i) continue;
                    const T dx = xj.x - xi.x + offx, dy = xj.y - xi.y + offy, dz = xj.z - xi.z + offz;
                    if (dx * dx + dy * dy + dz * dz < R2) {
                        if (count < kUfCap) row[count] = (int)((unsigned)j | (code << kUfShift));
                        ++count;
                    }
                }
            }
        }
    }
    b.uf_cnt[i] = count;
    if (count > kUfCap) atomicOr(&st.err, NEFE_ERR_NBR_OVERFLOW);
}
template <typename T>
__global__ void __launch_bounds__(kTile) k_uflist(Bufs b) {
    NEFE_FOR_TILES(b, uflist_tile<T>(b, tile));
}

// Fixed-point accumulation of the UF pair sums (order independent, so the unsorted rows give
// bitwise reproducible forces): 2^-32 units in the FP32 kernel, 2^-40 in the FP64 kernel.
template <typename T> struct UfFix;
template <> struct UfFix<float> {
    __device__ static long long to(float v) { return __float2ll_rn(v * 4294967296.0f); }
    __device__ static float from(long long q) { return (float)((double)q * 0x1p-32); }
};
template <> struct UfFix<double> {
    __device__ static long long to(double v) { return __double2ll_rn(v * 0x1p40); }
    __device__ static double from(long long q) { return (double)q * 0x1p-40; }
};
__device__ __forceinline__ float xexpm1(float v) { return expm1f(v); }
__device__ __forceinline__ double xexpm1(double v) { return ::expm1(v); }
__device__ __forceinline__ float xlogf_acc(float v) { return logf(v); }
__device__ __forceinline__ double xlogf_acc(double v) { return ::log(v); }

// Per step (or stateless): UF force and energy of each atom of a UF system from its row.
// Each pair is seen from both ends: half its energy and virial per end, the full force.
// The energy goes to U_int (pot = UF) or to the FL reference energy U_E (UF reference); the
// virial enters the pressure only when the UF term is U_int.
template <typename T, int MODE>
__global__ void __launch_bounds__(kTile) k_uf(Bufs b) {
    using T4 = typename V4<T>::t;
    __shared__ T4 soff[125];
    const int tile = b.uf_tiles ? b.uf_tiles[blockIdx.x] : (int)blockIdx.x;
    const TileAtom ta = tile_of(b, tile);
    const DevSys& S = b.sys[ta.sys];
    DevState& st = b.st[ta.sys];
    if (S.uf_mode == UF_NONE) return;            // uniform over the block
    if (threadIdx.x < 125) {
        const int c = threadIdx.x;
        const int ox = c % 5 - 2, oy = (c / 5) % 5 - 2, oz = c / 25 - 2;
        soff[c] = mk4((T)ox * pick<T>(st.h[0], st.h_f[0]), (T)oy * pick<T>(st.h[1], st.h_f[1]),
                      (T)oz * pick<T>(st.h[2], st.h_f[2]), (T)0);
    }
    __syncthreads();
    const T pk = pick<T>(S.uf_pk, S.uf_pk_f), is2 = pick<T>(S.uf_is2, S.uf_is2_f);
    const T rc2 = pick<T>(S.uf_rc2, S.uf_rc2_f), shift = pick<T>(S.uf_shift, S.uf_shift_f);
    long long q[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};   // f xyz, energy, virial xx yy zz xy xz yz
    const bool valid = (int)threadIdx.x < ta.count;
    const int i = ta.first + threadIdx.x;
    if (valid) {
        const T4* X = reinterpret_cast<const T4*>(b.xs);
        const T4 xi = X[i];
        const int cnt = min(b.uf_cnt[i], kUfCap);
        const int* row = b.uf_nbr + (size_t)i * kUfCap;
        for (int a = 0; a < cnt; ++a) {
            const unsigned e = (unsigned)row[a];
            if (!NEFE_IN_RANGE(e & kUfMask, b.ntot, &st.err)) continue;
            const T4 xj = X[e & kUfMask];
            const T4 oh = soff[e >> kUfShift];
            const T dx = (xj.x - xi.x) + oh.x, dy = (xj.y - xi.y) + oh.y, dz = (xj.z - xi.z) + oh.z;
            const T r2 = dx * dx + dy * dy + dz * dz;
            if (!(r2 < rc2)) continue;
            const T xx = r2 * is2;
            const T u = -pk * xlogf_acc(-xexpm1(-xx)) - shift;
            const T c = (T)2 * pk * is2 / xexpm1(xx);      // force on j along d: c d; on i: -c d
            const T hc = (T)0.5 * c;
            q[0] += UfFix<T>::to(-c * dx);
            q[1] += UfFix<T>::to(-c * dy);
            q[2] += UfFix<T>::to(-c * dz);
            q[3] += UfFix<T>::to((T)0.5 * u);
            q[4] += UfFix<T>::to(hc * dx * dx);
            q[5] += UfFix<T>::to(hc * dy * dy);
            q[6] += UfFix<T>::to(hc * dz * dz);
            q[7] += UfFix<T>::to(hc * dx * dy);
            q[8] += UfFix<T>::to(hc * dx * dz);
            q[9] += UfFix<T>::to(hc * dy * dz);
        }
    }
    T v[10];
#pragma unroll
    for (int k = 0; k < 10; ++k) v[k] = UfFix<T>::from(q[k]);
    if (valid) {
        if (MODE == FM_FORCES) {
            const size_t N = b.ntot;
            b.f_out[i] = (double)v[0]; b.f_out[N + i] = (double)v[1]; b.f_out[2 * N + i] = (double)v[2];
            if (b.e_atom) b.e_atom[i] = (double)v[3];
        } else {
            reinterpret_cast<T4*>(b.uf_F)[i] = mk4(v[0], v[1], v[2], v[3]);
        }
    }
    long long* acc = b.acc + (size_t)ta.sys * ACC_N * kSlots;
    if (S.uf_mode == UF_INT) {
        T red[8] = {v[3], (T)0, v[4], v[5], v[6], v[7], v[8], v[9]};   // U_int, (U_E), virial
        block_sum_to_acc<T, 8>(red, acc, ACC_UINT, &st.err);
    } else {
        T red[1] = {v[3]};
        block_sum_to_acc<T, 1>(red, acc, ACC_UREF, &st.err);
    }
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
    if (blockIdx.x == S.tile0 && threadIdx.x == 0) {
        for (int k = 0; k < 3; ++k) { st.ncell[k] = n3[k]; st.h[k] = h[k]; st.hb[k] = h[k]; }
        refresh_box_f(st);
    }
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
// Half kick + drift.  mode 0 (setup): mirror and noise only.
// x = anchor + dhi + dlo; per step the displacement grows by dt phi v + (s - 1) x (affine
// box drift).  In the FP32 path (dhi, dlo) is a compensated pair: a two-sum keeps the
// rounding error of every increment in dlo.
// ------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void comp_add(T& hi, T& lo, T d) {
    if constexpr (sizeof(T) == 8) {
        hi += d;
    } else {
        const T s = hi + d;
        const T bp = s - hi;
        const T err = (hi - (s - bp)) + (d - bp);
        lo += err;
        const T h2 = s + lo;
        lo = lo - (h2 - s);
        hi = h2;
    }
}

// Drift of atom i by its half-kicked velocity vk (move), its mirror, the displacement test (sets
// *flag) and the thermostat noise of step kstep (stored, and returned in z).  dh, dl: the atom's
// displacement, updated in place.  Shared by k_kick_drift and by the epilogue that moves the
// atoms for the next step (systems without a barostat), so both do the same operations.
// xa: the atom's mirror at the last build (loaded by the caller together with its other operands).
// any: the context-wide word that records that some system's flag was set (or NULL).
template <typename T>
__device__ __forceinline__ void drift_atom(const Bufs& b, const DevSys& S, const DevState& st, int i,
                                           const typename V4<T>::t& xa, const T (&vk)[3], bool move,
                                           T (&dh)[3], T (&dl)[3], int flag_set, int* flag, int* any,
                                           unsigned long long kstep, T (&z)[3]) {
    using T4 = typename V4<T>::t;
    const size_t N = b.ntot;
    T* DH = reinterpret_cast<T*>(b.dhi);
    T* DL = reinterpret_cast<T*>(b.dlo);
    const T xav[3] = {xa.x, xa.y, xa.z};
    const bool scaled = st.scaled != 0, hmoved = st.hmoved != 0;
    int4 q = make_int4(0, 0, 0, 0);
    if (scaled || hmoved) q = b.q[i];
    const int qa[3] = {q.x, q.y, q.z};
    if (move) {
        const T dt = pick<T>(b.dt, S.dt_f);
        for (int k = 0; k < 3; ++k) {
            T d = dt * pick<T>(st.phi[k], st.phi_f[k]) * vk[k];
            if (scaled) {   // (s - 1) x with x = xa + q hb + displacement
                const T xk = xav[k] + (T)qa[k] * pick<T>(st.hb[k], st.hb_f[k]) + dh[k];
                d += pick<T>(st.s[k] - 1.0, st.sm1_f[k]) * xk;
            }
            comp_add<T>(dh[k], dl[k], d);
            DH[k * N + i] = dh[k];
            if constexpr (sizeof(T) == 4) DL[k * N + i] = dl[k];
        }
    }
    T m[3];
    for (int k = 0; k < 3; ++k) {
        m[k] = xav[k] + (dh[k] + dl[k]);
        if (hmoved) m[k] -= (T)qa[k] * (pick<T>(st.h[k], st.h_f[k]) - pick<T>(st.hb[k], st.hb_f[k]));
    }
    reinterpret_cast<T4*>(b.xs)[i] = mk4(m[0], m[1], m[2], (T)0);
    T dd2 = 0;
    for (int k = 0; k < 3; ++k) {
        const T dd = hmoved ? m[k] - xav[k] * pick<T>(st.h[k] / st.hb[k], st.rho_f[k]) : dh[k] + dl[k];
        dd2 += dd * dd;
    }
    if (dd2 > pick<T>(st.thr2, st.thr2_f) && !flag_set) {
        atomicOr(flag, 1);
        if (any) atomicOr(any, 1);
    }
    z[0] = z[1] = z[2] = (T)0;
    if (S.thermo) {
        Noise<T>::xi3(S.seed, (uint64_t)S.rng_id, (uint64_t)kstep, (uint64_t)(i - S.off), z);
        reinterpret_cast<T4*>(b.xi)[i] = mk4(z[0], z[1], z[2], (T)0);
    }
}

// skip: systems without a barostat were already kicked and moved by the previous step's
// epilogue (k_finish with fuse), so their tiles return at once.
template <typename T>
__global__ void __launch_bounds__(kTile) k_kick_drift(Bufs b, int mode, int skip) {
    using T4 = typename V4<T>::t;
    const TileAtom ta = tile_of(b, blockIdx.x);
    const DevSys& S = b.sys[ta.sys];
    DevState& st = b.st[ta.sys];
    if (skip && S.baro == BARO_NONE) return;     // uniform over the block (one system per tile)
    T xs_sum[3] = {(T)0, (T)0, (T)0};
    if ((int)threadIdx.x < ta.count) {
        const int i = ta.first + threadIdx.x;
        const size_t N = b.ntot;
        T* V = reinterpret_cast<T*>(b.v);
        const T* DH = reinterpret_cast<const T*>(b.dhi);
        const T* DL = reinterpret_cast<const T*>(b.dlo);
        const T4 xa = reinterpret_cast<const T4*>(b.xa)[i];
        T dh[3], dl[3], vk[3] = {(T)0, (T)0, (T)0};
        for (int k = 0; k < 3; ++k) {
            dh[k] = DH[k * N + i];
            if constexpr (sizeof(T) == 4) dl[k] = DL[k * N + i]; else dl[k] = (T)0;
        }
        if (mode == 1) {
            const T4 F = reinterpret_cast<const T4*>(b.F)[i];
            const T fv[3] = {F.x, F.y, F.z};
            const T ck = pick<T>(S.ckick, S.ckick_f);
            for (int k = 0; k < 3; ++k) {
                vk[k] = V[k * N + i] + ck * fv[k];
                V[k * N + i] = vk[k];
            }
        }
        drift_atom<T>(b, S, st, i, xa, vk, mode == 1, dh, dl, st.rebuild, &st.rebuild, b.any_rebuild,
                      (unsigned long long)st.k,
                      xs_sum);
    }
    block_sum_to_acc<T, 3>(xs_sum, b.acc + (size_t)ta.sys * ACC_N * kSlots, ACC_XI, &st.err);
}

// ------------------------------------------------------------------------------------
// Stillinger-Weber terms for one edge of length r (A):
//   phi = eps A (B s^-p - s^-q) exp(1/(s - a)),  g = exp(gamma/(s - a)),  s = r/sigma,
// with dphi/dr and dg/dr.
// ------------------------------------------------------------------------------------
// Distance (in sigma) below the cutoff a inside which an edge is treated as cut off: there
// exp(1/(s - a)) and exp(gamma/(s - a)) underflow to 0 anyway, and 1/(s - a) would overflow
// (0 * inf = NaN) when s rounds onto a.
template <typename T> __device__ __forceinline__ T cut_eps() { return sizeof(T) == 4 ? (T)1e-5 : (T)1e-12; }

template <typename T>
__device__ __forceinline__ void sw_edge(const SWc<T>& P, T r, T& phi, T& dphi, T& g, T& dg) {
    const T s = r * P.inv_sig;
    if (!(s < P.s_act) || !(s - P.a < -cut_eps<T>())) {
        phi = dphi = g = dg = (T)0;
        return;
    }
    const T id = xrcp(s - P.a);
    const T e1 = xexp(id);
    g = xexp(P.gam * id);
    T rp, rq;
    if (P.int_pq) {
        const T is2 = xrcp(s * s);
        rp = is2 * is2;
        rq = (T)1;
    } else {
        rp = xpow(s, -P.p);
        rq = xpow(s, -P.q);
    }
    const T poly = P.B * rp - rq;
    phi = P.epsA * poly * e1;
    dphi = P.epsA * e1 * ((-P.p * P.B * rp + P.q * rq) * xrcp(s) - poly * id * id) * P.inv_sig;
    dg = -g * P.gam * id * id * P.inv_sig;
}

// Derivatives of one pair term phi2(r) with respect to A, B, p, q, a (sigma, eps fixed):
// phi2 = eps A (B s^-p - s^-q) e,  e = exp(1/(s - a)).
template <typename T>
__device__ __forceinline__ void sw_pair_pgrad(const SWc<T>& P, T r, T out[5]) {
    const T s = r * P.inv_sig;
    if (!(s < P.s_act) || !(s - P.a < -cut_eps<T>())) {
        for (int k = 0; k < 5; ++k) out[k] = (T)0;
        return;
    }
    const T id = xrcp(s - P.a);
    const T e1 = xexp(id);
    const T ls = xlog(s);
    const T rp = xpow(s, -P.p), rq = xpow(s, -P.q);
    const T ea = P.eps * P.A * e1;
    const T phi = ea * (P.B * rp - rq);
    out[0] = phi / P.A;                 // d/dA
    out[1] = ea * rp;                   // d/dB
    out[2] = -ea * P.B * rp * ls;       // d/dp
    out[3] = ea * rq * ls;              // d/dq
    out[4] = phi * id * id;             // d/da (pair exponent)
}

// Force pass A.  L lanes per atom, 128/L atoms per block.
//  1. The lanes compact the atom's Verlet row into its in-cutoff shell: (d, r^2) in shared
//     memory, the neighbour indices in shj (ended by -1 when shorter than kShell).
//  2. Lane a owns shell edge a: pair term (full force on i, half the energy), g, dg/dr and the
//     unit vector u_a.
//  3. Lane a sums over the other edges b the force that triplet (i; a, b) exerts on the leg
//     atom j_a,  F_a(b) = -t1 u_b + (t1 c - t2) u_a  with  c = u_a.u_b,
//     t1 = 2 eps lambda (c - c0) g_a g_b / r_a,  t2 = eps lambda (c - c0)^2 g_b (dg/dr)_a,
//     and stores the leg force L_a = sum_b F_a(b) in shd[i][a] for pass B.  Atom i gets -L_a
//     (the three forces of a triplet sum to zero) and half of h(i; a, b) per ordered pair.
// Each ordered pair costs ~14 flops and every triplet force is computed exactly once.
// P[i] = (pair + own triplet force, atom energy); block sums of energy and virial (and, with
// want_grad, of dE/d(A, B, p, q, a, lambda3, gamma)).
template <typename T, int L>
__global__ void __launch_bounds__(kTile) k_edges(Bufs b) {
    using T4 = typename V4<T>::t;
    constexpr int G = kTile / L;
    // rows padded by one entry: the groups of a warp then start on different banks
    __shared__ T4 sh_u[G][kShell + 1];     // (d, r^2) after compaction, then (u, r)
    __shared__ T sh_g[G][kShell + 1];
    __shared__ T sh_dg[G][kShell + 1];
    __shared__ T sh_id[G][kShell + 1];     // 1/(s - a), parameter gradients only
    __shared__ T4 soff[27];

    const int tile = blockIdx.x / L + b.tile_base, part = blockIdx.x % L;
    const TileAtom ta = tile_of(b, tile);
    const DevSys& S = b.sys[ta.sys];
    DevState& st = b.st[ta.sys];
    if (S.pot != POT_SW) return;                 // uniform over the block
    const SWc<T> P = reinterpret_cast<const SWc<T>*>(b.swc)[S.prm];
    const int lane = threadIdx.x % L, grp = threadIdx.x / L;
    const int lbase = ((threadIdx.x & 31) / L) * L;
    const unsigned gmask = (L == 32) ? 0xffffffffu : (((1u << L) - 1u) << lbase);
    offset_table<T>(soff, pick<T>(st.h[0], st.h_f[0]), pick<T>(st.h[1], st.h_f[1]), pick<T>(st.h[2], st.h_f[2]));
    const int ia = part * G + grp;
    const bool valid = ia < ta.count;
    const int i = ta.first + ia;

    T fx = 0, fy = 0, fz = 0, en = 0;
    T w0 = 0, w1 = 0, w2 = 0, w3 = 0, w4 = 0, w5 = 0;
    T gth[7] = {(T)0, (T)0, (T)0, (T)0, (T)0, (T)0, (T)0};   // dE/d(A, B, p, q, a, lambda3, gamma)
    const bool grad = b.want_grad != 0;
    if (valid) {
        const T4 xi = reinterpret_cast<const T4*>(b.xs)[i];
        const int ci = min(b.cnt[i], b.cap);
        T4* Fl = reinterpret_cast<T4*>(b.shd) + (size_t)i * kShell;
        int* Sj = b.shj + (size_t)i * kShell;
        // 1. compaction, NB row entries per lane in flight (row loads, then position gathers)
        constexpr int NB = (24 + L - 1) / L;
        int m = 0;
        for (int base = 0; base < ci; base += NB * L) {
            int e[NB];
            T4 xj[NB];
#pragma unroll
            for (int u = 0; u < NB; ++u) {
                const int sidx = base + u * L + lane;
                e[u] = sidx < ci ? b.nbr[nbr_at(b, i, sidx)] : 0;
                if (!NEFE_IN_RANGE(e[u] & (int)kIndexMask, b.ntot, &st.err)) e[u] = i;
            }
#pragma unroll
            for (int u = 0; u < NB; ++u)
                if (base + u * L + lane < ci) xj[u] = reinterpret_cast<const T4*>(b.xs)[e[u] & (int)kIndexMask];
#pragma unroll
            for (int u = 0; u < NB; ++u) {
                const int sidx = base + u * L + lane;
                bool in = false;
                T dx = 0, dy = 0, dz = 0, r2 = 0;
                if (sidx < ci) {
                    const T4 oh = soff[(unsigned)e[u] >> kCodeShift];
                    dx = (xj[u].x - xi.x) + oh.x;
                    dy = (xj[u].y - xi.y) + oh.y;
                    dz = (xj[u].z - xi.z) + oh.z;
                    r2 = dx * dx + dy * dy + dz * dz;
                    in = r2 < P.act2;
                }
                const unsigned bal = __ballot_sync(gmask, in);
                if (in) {
                    const int pos = m + __popc(bal & ((1u << (threadIdx.x & 31)) - 1u));
                    if (pos < kShell) {
                        sh_u[grp][pos] = mk4(dx, dy, dz, r2);
                        Sj[pos] = e[u] & (int)kIndexMask;
                    }
                }
                m += __popc(bal);
            }
        }
        if (m > kShell) {
            if (lane == 0) atomicOr(&st.err, NEFE_ERR_SHELL_OVERFLOW);
            m = kShell;
        }
        if (lane == 0 && m < kShell) Sj[m] = -1;
        __syncwarp(gmask);
        // 2. edges: pair terms, g, dg, unit vectors
        for (int a = lane; a < m; a += L) {
            const T4 d = sh_u[grp][a];
            const T ir = xrsqrt(d.w);
            const T r = d.w * ir;
            T phi, dphi, g, dg;
            sw_edge<T>(P, r, phi, dphi, g, dg);
            const T c = dphi * ir;
            fx += c * d.x; fy += c * d.y; fz += c * d.z;
            en += (T)0.5 * phi;
            const T hc = (T)-0.5 * c;
            w0 += hc * d.x * d.x; w1 += hc * d.y * d.y; w2 += hc * d.z * d.z;
            w3 += hc * d.x * d.y; w4 += hc * d.x * d.z; w5 += hc * d.y * d.z;
            sh_u[grp][a] = mk4(d.x * ir, d.y * ir, d.z * ir, r);
            sh_g[grp][a] = g;
            sh_dg[grp][a] = dg;
            if (grad) {   // each pair is seen from both ends: half of each derivative
                T pg[5];
                sw_pair_pgrad<T>(P, r, pg);
                for (int k = 0; k < 5; ++k) gth[k] += (T)0.5 * pg[k];
                const T den = r * P.inv_sig - P.a;
                sh_id[grp][a] = den < -cut_eps<T>() ? xrcp(den) : (T)0;
            }
        }
        __syncwarp(gmask);
        // 3. leg forces
        for (int a = lane; a < m; a += L) {
            const T4 ua = sh_u[grp][a];
            const T ga = sh_g[grp][a];
            const T k1 = (T)2 * P.epslam * ga * xrcp(ua.w);
            const T k2 = P.epslam * sh_dg[grp][a];
            T ax = 0, ay = 0, az = 0, cc = 0, eh = 0, e1 = 0, e2 = 0;
            for (int bb = 0; bb < m; ++bb) {
                if (bb == a) continue;
                const T4 ub = sh_u[grp][bb];
                const T gb = sh_g[grp][bb];
                const T c = ua.x * ub.x + ua.y * ub.y + ua.z * ub.z;
                const T dc = c - P.c0;
                const T s1 = dc * gb;
                const T t1 = k1 * s1;
                ax += t1 * ub.x; ay += t1 * ub.y; az += t1 * ub.z;
                cc += t1 * c - k2 * dc * s1;
                const T hb = dc * s1;                    // (c - c0)^2 g_b
                eh += hb;
                if (grad) {
                    const T idb = sh_id[grp][bb];
                    e1 += hb * idb;
                    e2 += hb * idb * idb;
                }
            }
            const T lx = cc * ua.x - ax, ly = cc * ua.y - ay, lz = cc * ua.z - az;
            Fl[a] = mk4(lx, ly, lz, (T)0);
            fx -= lx; fy -= ly; fz -= lz;
            const T hsum = (T)0.5 * P.epslam * ga * eh;  // half of every triplet (i; a, b), b != a
            en += hsum;
            const T dx = ua.x * ua.w, dy = ua.y * ua.w, dz = ua.z * ua.w;
            w0 += dx * lx; w1 += dy * ly; w2 += dz * lz;
            w3 += (T)0.5 * (dx * ly + dy * lx);
            w4 += (T)0.5 * (dx * lz + dz * lx);
            w5 += (T)0.5 * (dy * lz + dz * ly);
            if (grad) {
                const T ida = sh_id[grp][a];
                const T hh = (T)0.5 * P.epslam * ga;
                gth[4] += hh * P.gam * (ida * ida * eh + e2);
                gth[5] += (T)0.5 * P.eps * ga * eh;
                gth[6] += hh * (ida * eh + e1);
            }
        }
        // the atom's force, energy and virial (summed over its lanes); pass B adds the energy
        // and virial to its block sums, so this pass has no block reduction
        T v[10] = {fx, fy, fz, en, w0, w1, w2, w3, w4, w5};
#pragma unroll
        for (int o = L / 2; o > 0; o >>= 1)
#pragma unroll
            for (int k = 0; k < 10; ++k) v[k] += __shfl_xor_sync(gmask, v[k], o);
        if (lane == 0) {
            T4* Pa = reinterpret_cast<T4*>(b.P);
            Pa[i] = mk4(v[0], v[1], v[2], v[3]);
            Pa[b.ntot + 2 * (size_t)i] = mk4(v[4], v[5], v[6], v[7]);
            Pa[b.ntot + 2 * (size_t)i + 1] = mk4(v[8], v[9], (T)0, (T)0);
            b.shn[i] = m;
        }
    }
    if (grad) block_sum_to_acc<T, 7>(gth, b.acc + (size_t)ta.sys * ACC_N * kSlots, ACC_DTH, &st.err);
}

// Force pass A, one thread per atom (64-thread blocks, half a tile each), FP32: the same
// three phases as k_edges with no lane coordination (no ballots, no idle lanes while another
// holds edges).  The shell is a column per thread: its first kShell1Shared entries in shared
// memory (20 bytes each; this table bounds the occupancy, so it is sized for the typical
// shell), the rest up to kShell1 in a per-atom spill area in global memory (b.spill; without
// one the capacity is kShell1Shared).  Loop counters are equal across a warp, so the choice
// between the two places is uniform.
constexpr int kShell1Shared = 8;
constexpr int kShell1 = kShell1Shared + kSpill1;
constexpr int kEdges1Threads = 64;

// Scatter form of the force passes: pass A adds every leg force (and the atom's own force)
// into per-atom int32 accumulators (units of 2^-21 eV/A) with global reductions.  Integer
// addition is associative, so the result does not depend on the order in which the
// reductions arrive (bitwise reproducible), and no second pass has to find the legs again:
// a streaming epilogue (k_finish) reads and clears each atom's accumulator.  A term is
// rounded to 2^-22 eV/A; one above kLegLimit eV/A (whose sum over the terms an atom can
// receive could overflow int32) is dropped and flags the system.
// The x and y terms travel in one 64-bit reduction as y 2^32 + x (two's complement, modulo
// 2^64): integer addition is linear, so the 64-bit word accumulates Y 2^32 + X exactly, X and Y
// being the int32 sums.  Its low word is X; its high word is Y - 1 when X < 0 (the borrow), which
// the reader undoes (force_of_acc).  Two reductions per force instead of three.
constexpr float kLegScale = 2097152.0f;          // 2^21
constexpr float kLegLimit = 48.0f;
__device__ __forceinline__ void red_force(int* acc4, float x, float y, float z, unsigned* err) {
    if (!(fabsf(x) < kLegLimit && fabsf(y) < kLegLimit && fabsf(z) < kLegLimit)) {
        atomicOr(err, NEFE_ERR_NAN);
        return;
    }
    const long long px = __float2int_rn(x * kLegScale), py = __float2int_rn(y * kLegScale);
    const unsigned long long xy = ((unsigned long long)py << 32) + (unsigned long long)px;
    atomicAdd(reinterpret_cast<unsigned long long*>(acc4), xy);
    atomicAdd(acc4 + 2, __float2int_rn(z * kLegScale));
}

// The int32 sums (X, Y, Z) of an accumulator written by red_force.
__device__ __forceinline__ int3 force_of_acc(int4 q) {
    return make_int3(q.x, q.y + (q.x < 0 ? 1 : 0), q.z);
}

constexpr int kEdges1K1 = kShell1Shared;

// One work item of the thread-per-atom pass A: half a tile (64 atoms).  Every thread of the
// block calls it with the same item.
// Pass A for atom i (thread-per-atom): compaction of its Verlet row into the in-cutoff shell
// (column t of the shared shell table, entries past its K1 rows in the global spill area), pair
// terms, and the leg forces of the triplets centred on i (stored per shell edge, or in the
// scatter form added into the force accumulators, with the energy and virial added to red8).
// pos(j) returns atom j's mirror position (from global memory or a shared copy).
template <typename T, bool SCATTER, int NT, typename PosFn>
__device__ __forceinline__ void edges1_atom(const Bufs& b, const SWc<T>& P, DevState& st,
                                            const T* soff, int i, int t,
                                            typename V4<T>::t (*sh_u)[NT], T (*sh_r)[NT], int (*sh_j)[NT],
                                            PosFn pos, T (&red8)[8]) {
    using T4 = typename V4<T>::t;
    constexpr int K1 = kShell1Shared, KS = kShell1 - kShell1Shared;
    const T4 xi = pos(i);
    const int ci = min(b.cnt[i], b.cap);
    const int* row = b.nbr + (size_t)i * b.cap;
    T4* Fl = reinterpret_cast<T4*>(b.shd) + (size_t)i * kShell;
    int* Sj = b.shj + (size_t)i * kShell;
    T4* spu = b.spill ? reinterpret_cast<T4*>(b.spill) + (size_t)i * KS : nullptr;
    T* spr = b.spill ? reinterpret_cast<T*>(reinterpret_cast<T4*>(b.spill) + (size_t)b.ntot * KS) + (size_t)i * KS
                     : nullptr;
    const int capm = b.spill ? kShell1 : K1;
    auto put_u = [&](int a, T4 v) { if (a < K1) sh_u[a][t] = v; else spu[a - K1] = v; };
    auto get_u = [&](int a) -> T4 { return a < K1 ? sh_u[a][t] : spu[a - K1]; };
    auto put_r = [&](int a, T v) { if (a < K1) sh_r[a][t] = v; else spr[a - K1] = v; };
    auto get_r = [&](int a) -> T { return a < K1 ? sh_r[a][t] : spr[a - K1]; };
    // 1. compaction, four row entries in flight.  Interleaved rows (engine): one 16-byte load
    // per four entries, contiguous across the warp, and the row is padded to a multiple of 4
    // with entries that fail the distance test, so every entry of the last group is read
    // unguarded.  Row-major rows: one 16-byte load when the row capacity is a multiple of 4,
    // entries past ci not used.
    int m = 0;
    const bool il = b.nbr_il != 0;
    const bool row4 = (b.cap & 3) == 0;
    const int cend = il ? (ci + 3) & ~3 : ci;
    const int4* row_il = reinterpret_cast<const int4*>(b.nbr) + i;
    for (int base = 0; base < cend; base += 4) {
        int e[4];
        T4 xj[4];
        if (il) {
            const int4 r4 = row_il[(size_t)(base >> 2) * b.ntot];
            e[0] = r4.x; e[1] = r4.y; e[2] = r4.z; e[3] = r4.w;
        } else if (row4) {
            const int4 r4 = *reinterpret_cast<const int4*>(row + base);
            e[0] = r4.x; e[1] = r4.y; e[2] = r4.z; e[3] = r4.w;
        } else {
#pragma unroll
            for (int u = 0; u < 4; ++u) e[u] = (base + u < ci) ? row[base + u] : 0;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (!NEFE_IN_RANGE(e[u] & (int)kIndexMask, b.ntot, &st.err)) e[u] = i;
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (il || base + u < ci) xj[u] = pos(e[u] & (int)kIndexMask);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (!il && base + u >= ci) continue;
            const unsigned c = (unsigned)e[u] >> kCodeShift;
            const T dx = (xj[u].x - xi.x) + soff[c], dy = (xj[u].y - xi.y) + soff[32 + c],
                    dz = (xj[u].z - xi.z) + soff[64 + c];
            const T r2 = dx * dx + dy * dy + dz * dz;
            if (r2 < P.act2) {
                if (m < capm) {
                    put_u(m, mk4(dx, dy, dz, r2));
                    // the scatter form keeps the shell's atom indices next to it in shared memory
                    // (global only past its rows); the gather form publishes them for pass B
                    if (SCATTER && m < K1) sh_j[m][t] = e[u] & (int)kIndexMask;
                    else Sj[m] = e[u] & (int)kIndexMask;
                }
                ++m;
            }
        }
    }
    if (m > capm) {
        atomicOr(&st.err, NEFE_ERR_SHELL_OVERFLOW);
        m = capm;
    }
    if (!SCATTER && m < kShell) Sj[m] = -1;
    T fx = 0, fy = 0, fz = 0, en = 0;
    T w0 = 0, w1 = 0, w2 = 0, w3 = 0, w4 = 0, w5 = 0;
    // Moments of the shell: G = sum_b g_b, m1 = sum_b g_b u_b, M = sum_b g_b u_b u_b^T.  Every
    // sum over the partner edge b of a triplet (i; a, b) that the leg force needs is linear in
    // these, so the triplets of an atom cost O(m) instead of O(m^2) (see phase 3).
    T G = 0, m1x = 0, m1y = 0, m1z = 0, Mxx = 0, Myy = 0, Mzz = 0, Mxy = 0, Mxz = 0, Myz = 0;
    // 2. edges
    for (int a = 0; a < m; ++a) {
        const T4 d = get_u(a);
        const T ir = xrsqrt(d.w);
        const T r = d.w * ir;
        T phi, dphi, g, dg;
        sw_edge<T>(P, r, phi, dphi, g, dg);
        const T c = dphi * ir;
        fx += c * d.x; fy += c * d.y; fz += c * d.z;
        en += (T)0.5 * phi;
        const T hc = (T)-0.5 * c;
        w0 += hc * d.x * d.x; w1 += hc * d.y * d.y; w2 += hc * d.z * d.z;
        w3 += hc * d.x * d.y; w4 += hc * d.x * d.z; w5 += hc * d.y * d.z;
        const T ux = d.x * ir, uy = d.y * ir, uz = d.z * ir;
        put_u(a, mk4(ux, uy, uz, g));
        put_r(a, r);
        const T gx = g * ux, gy = g * uy, gz = g * uz;
        G += g; m1x += gx; m1y += gy; m1z += gz;
        Mxx += gx * ux; Myy += gy * uy; Mzz += gz * uz; Mxy += gx * uy; Mxz += gx * uz; Myz += gy * uz;
    }
    // 3. leg forces.  For edge a with c_b = u_a.u_b, over every partner b != a:
    //   S1 = sum g_b (c_b - c0) u_b = M u_a - c0 m1 - g_a (1 - c0) u_a,
    //   S2 = sum g_b (c_b - c0) c_b = u_a.M u_a - c0 u_a.m1 - g_a (1 - c0),
    //   S3 = sum g_b (c_b - c0)^2   = u_a.M u_a - 2 c0 u_a.m1 + c0^2 G - g_a (1 - c0)^2
    // (the sums over all b, minus the b = a term with c = 1).  The force the triplets (i; a, b)
    // exert on leg atom j_a is L_a = (k1 S2 - k2 S3) u_a - k1 S1 with k1 = 2 eps lambda g_a / r_a,
    // k2 = eps lambda dg_a/dr, and the atom's share of their energy is eps lambda g_a S3 / 2.
    const T c0 = P.c0, c02 = c0 * c0;
    for (int a = 0; a < m; ++a) {
        const T4 ua = get_u(a);
        const T ga = ua.w, ra = get_r(a);
        // dg/dr of edge a from g and r: -g gamma / (sigma (s - a)^2) (0 beyond the active cutoff)
        const T den = ra * P.inv_sig - P.a;
        const T ida = den < -cut_eps<T>() ? xrcp(den) : (T)0;
        const T dga = -ga * P.gam * ida * ida * P.inv_sig;
        const T k1 = (T)2 * P.epslam * ga * xrcp(ra);
        const T k2 = P.epslam * dga;
        const T Mux = Mxx * ua.x + Mxy * ua.y + Mxz * ua.z;
        const T Muy = Mxy * ua.x + Myy * ua.y + Myz * ua.z;
        const T Muz = Mxz * ua.x + Myz * ua.y + Mzz * ua.z;
        const T q = ua.x * Mux + ua.y * Muy + ua.z * Muz;
        const T pm = ua.x * m1x + ua.y * m1y + ua.z * m1z;
        const T self = ga * ((T)1 - c0);
        const T S2 = q - c0 * pm - self;
        const T S3 = q - (T)2 * c0 * pm + c02 * G - self * ((T)1 - c0);
        const T eh = S3;
        const T cc = k1 * S2 - k2 * S3;
        const T ax = k1 * (Mux - c0 * m1x - self * ua.x);
        const T ay = k1 * (Muy - c0 * m1y - self * ua.y);
        const T az = k1 * (Muz - c0 * m1z - self * ua.z);
        const T lx = cc * ua.x - ax, ly = cc * ua.y - ay, lz = cc * ua.z - az;
        if constexpr (SCATTER) red_force(b.lacc + 4 * (size_t)(a < K1 ? sh_j[a][t] : Sj[a]), lx, ly, lz, &st.err);
        else Fl[a] = mk4(lx, ly, lz, (T)0);
        fx -= lx; fy -= ly; fz -= lz;
        en += (T)0.5 * P.epslam * ga * eh;
        const T dx = ua.x * ra, dy = ua.y * ra, dz = ua.z * ra;
        w0 += dx * lx; w1 += dy * ly; w2 += dz * lz;
        w3 += (T)0.5 * (dx * ly + dy * lx);
        w4 += (T)0.5 * (dx * lz + dz * lx);
        w5 += (T)0.5 * (dy * lz + dz * ly);
    }
    if constexpr (SCATTER) {
        red_force(b.lacc + 4 * (size_t)i, fx, fy, fz, &st.err);
        if (b.e_atom) b.e_atom[i] = (double)en;
        red8[0] += en;
        red8[2] += w0; red8[3] += w1; red8[4] += w2; red8[5] += w3; red8[6] += w4; red8[7] += w5;
    } else {
        T4* Pa = reinterpret_cast<T4*>(b.P);
        Pa[i] = mk4(fx, fy, fz, en);
        Pa[b.ntot + 2 * (size_t)i] = mk4(w0, w1, w2, w3);
        Pa[b.ntot + 2 * (size_t)i + 1] = mk4(w4, w5, (T)0, (T)0);
    }
    b.shn[i] = m;
}

template <typename T, bool SCATTER>
__device__ __forceinline__ void edges1_item(const Bufs& b, int tile, int part, typename V4<T>::t (*sh_u)[kEdges1Threads],
                                            T (*sh_r)[kEdges1Threads], int (*sh_j)[kEdges1Threads],
                                            T* soff) {
    using T4 = typename V4<T>::t;
    constexpr int NT = kEdges1Threads;
    // 20 bytes per shell entry and thread (occupancy is bound by this table):
    constexpr int K1 = kShell1Shared, KS = kShell1 - kShell1Shared;
    const TileAtom ta = tile_of(b, tile);
    const DevSys& S = b.sys[ta.sys];
    DevState& st = b.st[ta.sys];
    if (S.pot != POT_SW) return;                 // uniform over the block
    const SWc<T> P = reinterpret_cast<const SWc<T>*>(b.swc)[S.prm];
    offset_rows<T>(soff, pick<T>(st.h[0], st.h_f[0]), pick<T>(st.h[1], st.h_f[1]), pick<T>(st.h[2], st.h_f[2]));
    const int t = threadIdx.x;
    const int ia = part * NT + t;
    T red8[8] = {(T)0, (T)0, (T)0, (T)0, (T)0, (T)0, (T)0, (T)0};   // scatter form: energy, -, virial
    if (ia < ta.count) {
        const T4* X = reinterpret_cast<const T4*>(b.xs);
        edges1_atom<T, SCATTER, kEdges1Threads>(b, P, st, soff, ta.first + ia, t, sh_u, sh_r, sh_j,
                                               [X](int j) { return X[j]; }, red8);
    }
    if constexpr (SCATTER) block_sum_to_acc<T, 8>(red8, b.acc + (size_t)ta.sys * ACC_N * kSlots, ACC_UINT, &st.err);
}

template <typename T, bool SCATTER>
__global__ void __launch_bounds__(kEdges1Threads, 16) k_edges1(Bufs b) {
    using T4 = typename V4<T>::t;
    __shared__ T4 sh_u[kEdges1K1][kEdges1Threads];   // (d, r^2) after compaction, then (u, g)
    __shared__ T sh_r[kEdges1K1][kEdges1Threads];    // r
    __shared__ int sh_j[SCATTER ? kEdges1K1 : 1][kEdges1Threads];   // shell atom indices (scatter form)
    __shared__ T soff[3 * 32];
    constexpr int IPT = kTile / kEdges1Threads;  // work items per tile
    edges1_item<T, SCATTER>(b, (int)blockIdx.x / IPT + b.tile_base, (int)blockIdx.x % IPT, sh_u, sh_r, sh_j, soff);
}

// Force pass B, L lanes per atom:
//   F_SW(i) = P(i) + sum_{j in shell(i)} L_j(i),
// L_j(i) being the leg force that the triplets centred on neighbour j exert on i, stored by
// pass A at the position of i in j's shell (found by scanning j's index list; shells are
// symmetric because both ends compute the same r^2 bit for bit).  Then, in FM_SETUP /
// FM_STEP: Einstein springs, lambda mixing, Langevin force (this step's noise with its
// per-system mean removed), second half kick and the kinetic sums.
template <typename T, int MODE>
__device__ __forceinline__ void finish_atom(const Bufs& b, const DevSys& S, const DevState& st, int i,
                                            const T (&f)[3], T e_i, bool write_e, const T (&pd)[3],
                                            const T (&pv)[3], const T (&pz)[3], const T* s_xm, T (&red)[14],
                                            bool keep, T (&vo)[3], T (&Fo)[3]);
template <typename T>
__device__ __forceinline__ void noise_mean(const Bufs& b, const DevSys& S, int sys, T* s_xm);
template <typename T>
__device__ __forceinline__ void noise_mean_staged(const DevSys& S, const long long (*xi)[kSlots], T* s_xm);

template <typename T, int MODE, int L>
__global__ void __launch_bounds__(kTile) k_gather(Bufs b) {
    using T4 = typename V4<T>::t;
    constexpr int G = kTile / L;
    const int tile = blockIdx.x / L + b.tile_base, part = blockIdx.x % L;
    __shared__ __align__(16) StagedSys sh;
    __shared__ long long s_xi[3][kSlots];
    __shared__ T s_xm[3];
    if (MODE != FM_FORCES) {   // the noise sums' slots, loaded with the descriptors
        const int sys = b.tile_sys[tile];
        const long long* xa = b.acc + (size_t)sys * ACC_N * kSlots + (size_t)ACC_XI * kSlots;
        for (int w = threadIdx.x; w < 3 * kSlots; w += blockDim.x) s_xi[w / kSlots][w % kSlots] = xa[w];
    }
    const TileAtom ta = stage_tile(b, tile, sh);
    const DevSys& S = sh.S;
    const DevState& st = sh.st;
    DevState& gst = b.st[ta.sys];
    if (MODE != FM_FORCES) noise_mean_staged<T>(S, s_xi, s_xm);
    __syncthreads();
    const int lane = threadIdx.x % L, grp = threadIdx.x / L;
    const int lbase = ((threadIdx.x & 31) / L) * L;
    const unsigned gmask = (L == 32) ? 0xffffffffu : (((1u << L) - 1u) << lbase);
    T red[14];
#pragma unroll
    for (int k = 0; k < 14; ++k) red[k] = (T)0;
    const int ia = part * G + grp;
    if (ia < ta.count) {
        const int i = ta.first + ia;
        const size_t N = b.ntot;
        T f[3] = {(T)0, (T)0, (T)0}, e_i = 0;
        // the epilogue's own-atom operands are loaded first, so their latency overlaps the gather
        T pd[3] = {(T)0, (T)0, (T)0}, pv[3] = {(T)0, (T)0, (T)0}, pz[3] = {(T)0, (T)0, (T)0};
        if (MODE != FM_FORCES && lane == 0) {
            if (S.springs) {
                const T4 d0 = reinterpret_cast<const T4*>(b.sd0)[i];
                const T* DH = reinterpret_cast<const T*>(b.dhi);
                const T* DL = reinterpret_cast<const T*>(b.dlo);
                pd[0] = d0.x; pd[1] = d0.y; pd[2] = d0.z;
                for (int k = 0; k < 3; ++k) {
                    pd[k] += DH[k * N + i];
                    if constexpr (sizeof(T) == 4) pd[k] += DL[k * N + i];
                }
            }
            const T* V = reinterpret_cast<const T*>(b.v);
            pv[0] = V[i]; pv[1] = V[N + i]; pv[2] = V[2 * N + i];
            if (S.thermo) {
                const T4 z = reinterpret_cast<const T4*>(b.xi)[i];
                pz[0] = z.x; pz[1] = z.y; pz[2] = z.z;
            }
        }
        if (S.pot == POT_SW) {
            const T4* Fl = reinterpret_cast<const T4*>(b.shd);
            const int m = b.shn[i];
            // NB shell entries per lane in flight: neighbour index, the first 8 entries of the
            // neighbour's index list (one 32-byte sector), then the leg force
            constexpr int NB = L >= 2 ? 1 : 2;
            for (int base = 0; base < m; base += NB * L) {
                int jj[NB], pos[NB];
                int4 q0[NB], q1[NB];
                if constexpr (NB == 2 && L == 1) {   // both entries with one 8-byte load (rows are 128 bytes)
                    const int2 j2 = *reinterpret_cast<const int2*>(b.shj + (size_t)i * kShell + base);
                    jj[0] = j2.x;
                    jj[NB - 1] = base + 1 < m ? j2.y : -1;
                } else {
#pragma unroll
                    for (int u = 0; u < NB; ++u) {
                        const int a = base + u * L + lane;
                        jj[u] = a < m ? b.shj[(size_t)i * kShell + a] : -1;
                    }
                }
#pragma unroll
                for (int u = 0; u < NB; ++u)
                    if (jj[u] >= 0 && !NEFE_IN_RANGE(jj[u], b.ntot, &gst.err)) jj[u] = -1;
#pragma unroll
                for (int u = 0; u < NB; ++u) {
                    if (jj[u] >= 0) {
                        const int4* Sq = reinterpret_cast<const int4*>(b.shj + (size_t)jj[u] * kShell);
                        q0[u] = Sq[0];
                        q1[u] = Sq[1];
                    }
                }
#pragma unroll
                for (int u = 0; u < NB; ++u) {
                    pos[u] = -1;
                    if (jj[u] < 0) continue;
                    const int w8[8] = {q0[u].x, q0[u].y, q0[u].z, q0[u].w, q1[u].x, q1[u].y, q1[u].z, q1[u].w};
                    bool ended = false;
#pragma unroll
                    for (int t = 0; t < 8; ++t) {
                        if (!ended && pos[u] < 0) {
                            if (w8[t] == i) pos[u] = t;
                            else if (w8[t] < 0) ended = true;
                        }
                    }
                    if (pos[u] < 0 && !ended) {          // i beyond the first 8 entries of j's shell
                        const int* Sj = b.shj + (size_t)jj[u] * kShell;
                        for (int t = 8; t < kShell; ++t) {
                            const int q = Sj[t];
                            if (q == i) { pos[u] = t; break; }
                            if (q < 0) break;
                        }
                    }
                }
                T4 lf[NB];
#pragma unroll
                for (int u = 0; u < NB; ++u)
                    if (pos[u] >= 0) lf[u] = Fl[(size_t)jj[u] * kShell + pos[u]];
#pragma unroll
                for (int u = 0; u < NB; ++u)
                    if (pos[u] >= 0) { f[0] += lf[u].x; f[1] += lf[u].y; f[2] += lf[u].z; }
            }
#pragma unroll
            for (int o = L / 2; o > 0; o >>= 1) {
                f[0] += __shfl_xor_sync(gmask, f[0], o);
                f[1] += __shfl_xor_sync(gmask, f[1], o);
                f[2] += __shfl_xor_sync(gmask, f[2], o);
            }
            const T4* Pa = reinterpret_cast<const T4*>(b.P);
            const T4 p = Pa[i];
            f[0] += p.x; f[1] += p.y; f[2] += p.z; e_i = p.w;
            if (lane == 0) {
                const T4 wa = Pa[b.ntot + 2 * (size_t)i], wb = Pa[b.ntot + 2 * (size_t)i + 1];
                red[0] = e_i;
                red[2] = wa.x; red[3] = wa.y; red[4] = wa.z; red[5] = wa.w; red[6] = wb.x; red[7] = wb.y;
            }
        }
        T vo[3], Fo[3];
        if (lane == 0) finish_atom<T, MODE>(b, S, st, i, f, e_i, true, pd, pv, pz, s_xm, red, false, vo, Fo);
    }
    block_sum_to_acc<T, 14>(red, b.acc + (size_t)ta.sys * ACC_N * kSlots, ACC_UINT, &gst.err);
}

// The epilogue of force pass B for atom i with SW (or zero) force f: the stateless output, or
// Einstein springs / UF force, lambda mixing, Langevin force with the per-system mean of this
// step's noise removed, second half kick, total force for the next step and the kinetic sums.
// pd: spring offset x - r0; pv: velocity; pz: noise of the step; s_xm: the per-system noise mean.
// keep: the velocity and total force are returned in vo, Fo instead of being stored (the caller
// goes on to the next step's kick and drift).
template <typename T, int MODE>
__device__ __forceinline__ void finish_atom(const Bufs& b, const DevSys& S, const DevState& st, int i,
                                            const T (&f)[3], T e_i, bool write_e, const T (&pd)[3],
                                            const T (&pv)[3], const T (&pz)[3], const T* s_xm, T (&red)[14],
                                            bool keep, T (&vo)[3], T (&Fo)[3]) {
    using T4 = typename V4<T>::t;
    const size_t N = b.ntot;
            if (MODE == FM_FORCES) {
                b.f_out[i] = (double)f[0]; b.f_out[N + i] = (double)f[1]; b.f_out[2 * N + i] = (double)f[2];
                if (b.e_atom && write_e) b.e_atom[i] = (double)e_i;
            } else {
                T fint[3] = {f[0], f[1], f[2]}, fe[3] = {(T)0, (T)0, (T)0};
                T u_int = 0, u_ref = 0;
                if (S.springs) {
                    const T d[3] = {pd[0], pd[1], pd[2]};
                    const T d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                    if (S.pot == POT_EINSTEIN) {
                        const T k_i = pick<T>(S.k_int, S.kint_f);
                        u_int = (T)0.5 * k_i * d2;
                        for (int k = 0; k < 3; ++k) fint[k] = -k_i * d[k];
                    }
                    const T k_e = pick<T>(S.k_E, S.kE_f);
                    u_ref = (T)0.5 * k_e * d2;
                    for (int k = 0; k < 3; ++k) fe[k] = -k_e * d[k];
                }
                if (S.uf_mode != UF_NONE) {     // UF force of this step (its energy is summed by k_uf)
                    const T4 fu = reinterpret_cast<const T4*>(b.uf_F)[i];
                    T* dst = S.uf_mode == UF_INT ? fint : fe;
                    dst[0] = fu.x; dst[1] = fu.y; dst[2] = fu.z;
                }
                T* V = reinterpret_cast<T*>(b.v);
                T v[3] = {pv[0], pv[1], pv[2]};
                const T si = pick<T>(st.scale_int, st.scale_int_f), se = pick<T>(st.scale_E, st.scale_E_f);
                T F[3];
                for (int k = 0; k < 3; ++k) F[k] = si * fint[k] + se * fe[k];
                if (S.thermo) {
                    const T zz[3] = {pz[0], pz[1], pz[2]};
                    const T amp = pick<T>(S.amp, S.amp_f), gam = pick<T>(S.gam, S.gam_f);
                    for (int k = 0; k < 3; ++k) F[k] += -gam * v[k] + amp * (zz[k] - s_xm[k]);
                }
                if (MODE == FM_STEP) {
                    const T ck = pick<T>(S.ckick, S.ckick_f);
                    for (int k = 0; k < 3; ++k) {
                        v[k] += ck * F[k];
                        if (!keep) V[k * N + i] = v[k];
                    }
                }
                for (int k = 0; k < 3; ++k) { vo[k] = v[k]; Fo[k] = F[k]; }
                if (!keep) reinterpret_cast<T4*>(b.F)[i] = mk4(F[0], F[1], F[2], (T)0);
                const T me = pick<T>(S.mass_e, S.mass_f);
                red[0] += u_int;
                red[1] = u_ref;
                red[8] = me * v[0] * v[0];
                red[9] = me * v[1] * v[1];
                red[10] = me * v[2] * v[2];
                red[11] = me * v[0] * v[1];
                red[12] = me * v[0] * v[2];
                red[13] = me * v[1] * v[2];
            }
}

// Per-system mean of this step's thermostat noise (the "zero yes" removal), from the
// fixed-point sums of k_kick_drift, into s_xm[3].  Threads 0..2 write; the caller syncs.
// The same mean from the noise sums' slots already copied to shared memory (3 x kSlots).
template <typename T>
__device__ __forceinline__ void noise_mean_staged(const DevSys& S, const long long (*xi)[kSlots], T* s_xm) {
    if (threadIdx.x < 3) {
        long long sum = 0;
        for (int sl = 0; sl < kSlots; ++sl) sum += xi[threadIdx.x][sl];
        if constexpr (sizeof(T) == 4) {
            const float hi = (float)(int)(sum >> 32);
            const float lo = (float)(unsigned)(sum & 0xffffffffLL) * 0x1p-32f;
            s_xm[threadIdx.x] = (hi + lo) * S.inv_n_f;
        } else {
            s_xm[threadIdx.x] = (T)((double)sum / kFix / (double)S.n);
        }
    }
}

template <typename T>
__device__ __forceinline__ void noise_mean(const Bufs& b, const DevSys& S, int sys, T* s_xm) {
    if (threadIdx.x < 3) {
        const long long* acc = b.acc + (size_t)sys * ACC_N * kSlots + (size_t)(ACC_XI + threadIdx.x) * kSlots;
        const long long sum = slot_sum(acc);
        if constexpr (sizeof(T) == 4) {   // sum 2^-32 / n from its 32-bit halves, FP32 only
            const float hi = (float)(int)(sum >> 32);
            const float lo = (float)(unsigned)(sum & 0xffffffffLL) * 0x1p-32f;
            s_xm[threadIdx.x] = (hi + lo) * S.inv_n_f;
        } else {
            s_xm[threadIdx.x] = (T)((double)sum / kFix / (double)S.n);
        }
    }
}

// Force pass B of the scatter form: one thread per atom reads and clears the atom's force
// accumulator (the pair, own-triplet and leg forces pass A added) and runs the epilogue.  The
// SW energy and virial were summed by pass A.
// fuse (FM_STEP, systems without a barostat): the epilogue goes straight on to the next step's
// first half kick, drift, mirror, displacement test and thermostat noise -- the work of
// k_kick_drift, which then skips these systems.  Nothing between the two reads or changes what
// that work uses (no barostat: the box, drift factors and rebuild threshold stay as they are),
// and the operations are the same ones, so the trajectory is bit for bit that of the unfused
// sequence.  The force of the step is not stored (the next half kick consumed it); the noise
// sums go to ACC_XIN and the rebuild flag to rebuild_next, which the next k_group moves into
// place.  The last step of every launch sequence runs unfused, so the state between calls is
// the usual one (positions and velocities at a full step).
template <typename T, int MODE>
__global__ void __launch_bounds__(kTile) k_finish(Bufs b, int fuse) {
    using T4 = typename V4<T>::t;
    const int tile = blockIdx.x + b.tile_base;
    __shared__ __align__(16) StagedSys sh;
    __shared__ long long s_xi[3][kSlots];
    __shared__ T s_xm[3];
    if (MODE != FM_FORCES) {   // the noise sums' slots, loaded with the descriptors
        const int sys = b.tile_sys[tile];
        const long long* xa = b.acc + (size_t)sys * ACC_N * kSlots + (size_t)ACC_XI * kSlots;
        for (int w = threadIdx.x; w < 3 * kSlots; w += blockDim.x) s_xi[w / kSlots][w % kSlots] = xa[w];
    }
    const TileAtom ta = stage_tile(b, tile, sh);
    const DevSys& S = sh.S;
    const DevState& st = sh.st;
    DevState& gst = b.st[ta.sys];
    if (MODE != FM_FORCES) noise_mean_staged<T>(S, s_xi, s_xm);
    __syncthreads();
    const bool fz = MODE == FM_STEP && fuse && S.baro == BARO_NONE;   // uniform over the block
    T red[14];
#pragma unroll
    for (int k = 0; k < 14; ++k) red[k] = (T)0;
    T zn[3] = {(T)0, (T)0, (T)0};
    if ((int)threadIdx.x < ta.count) {
        const int i = ta.first + threadIdx.x;
        const size_t N = b.ntot;
        // every operand is loaded before the first is used, so the loads are in flight together
        // (this kernel streams its operands; nothing else hides their latency)
        const bool sw = S.pot == POT_SW, springs = MODE != FM_FORCES && S.springs;
        const bool thermo = MODE != FM_FORCES && S.thermo;
        int4* a4 = reinterpret_cast<int4*>(b.lacc) + i;
        int4 q = make_int4(0, 0, 0, 0);
        T4 d0 = mk4((T)0, (T)0, (T)0, (T)0), z = d0;
        T dh[3] = {(T)0, (T)0, (T)0}, dl[3] = {(T)0, (T)0, (T)0}, pv[3] = {(T)0, (T)0, (T)0};
        if (sw) q = *a4;
        if (springs || fz) {
            const T* DH = reinterpret_cast<const T*>(b.dhi);
            const T* DL = reinterpret_cast<const T*>(b.dlo);
            if (springs) d0 = reinterpret_cast<const T4*>(b.sd0)[i];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                dh[k] = DH[k * N + i];
                if constexpr (sizeof(T) == 4) dl[k] = DL[k * N + i];
            }
        }
        if (MODE != FM_FORCES) {
            const T* V = reinterpret_cast<const T*>(b.v);
            pv[0] = V[i]; pv[1] = V[N + i]; pv[2] = V[2 * N + i];
        }
        if (thermo) z = reinterpret_cast<const T4*>(b.xi)[i];
        T4 xa = mk4((T)0, (T)0, (T)0, (T)0);
        if (fz) xa = reinterpret_cast<const T4*>(b.xa)[i];
        if (sw) *a4 = make_int4(0, 0, 0, 0);
        const T pd[3] = {d0.x + dh[0] + dl[0], d0.y + dh[1] + dl[1], d0.z + dh[2] + dl[2]};
        const T pz[3] = {z.x, z.y, z.z};
        const T inv = (T)(1.0 / (double)kLegScale);
        const int3 fq = force_of_acc(q);
        const T f[3] = {(T)fq.x * inv, (T)fq.y * inv, (T)fq.z * inv};
        T vo[3], Fo[3];
        finish_atom<T, MODE>(b, S, st, i, f, (T)0, false, pd, pv, pz, s_xm, red, fz, vo, Fo);
        if (fz) {
            // the next step's first half kick (the force of this step, Langevin term included)
            T* V = reinterpret_cast<T*>(b.v);
            const T ck = pick<T>(S.ckick, S.ckick_f);
            T vk[3];
            for (int k = 0; k < 3; ++k) {
                vk[k] = vo[k] + ck * Fo[k];
                V[k * N + i] = vk[k];
            }
            drift_atom<T>(b, S, st, i, xa, vk, true, dh, dl, 0, &gst.rebuild_next,
                          b.any_rebuild ? b.any_rebuild + 1 : nullptr, (unsigned long long)st.k + 1ULL,
                          zn);
        }
    }
    block_sum_to_acc<T, 14>(red, b.acc + (size_t)ta.sys * ACC_N * kSlots, ACC_UINT, &gst.err);
    if (fz) block_sum_to_acc<T, 3>(zn, b.acc + (size_t)ta.sys * ACC_N * kSlots, ACC_XIN, &gst.err);
}

// FP64 positions and velocities for output, and replacement from FP64 input.
template <typename T>
__global__ void __launch_bounds__(kTile) k_materialize(Bufs b, double* x, double* v) {
    const TileAtom ta = tile_of(b, blockIdx.x);
    if ((int)threadIdx.x >= ta.count) return;
    const int i = ta.first + threadIdx.x;
    const size_t N = b.ntot;
    const T* DH = reinterpret_cast<const T*>(b.dhi);
    const T* DL = reinterpret_cast<const T*>(b.dlo);
    const T* V = reinterpret_cast<const T*>(b.v);
    for (int k = 0; k < 3; ++k) {
        if (x) {
            double d = (double)DH[k * N + i];
            if constexpr (sizeof(T) == 4) d += (double)DL[k * N + i];
            x[k * N + i] = b.x[k * N + i] + d;
        }
        if (v) v[k * N + i] = (double)V[k * N + i];
    }
}

template <typename T>
__global__ void __launch_bounds__(kTile) k_inject(Bufs b, const double* x, const double* v) {
    const TileAtom ta = tile_of(b, blockIdx.x);
    if ((int)threadIdx.x >= ta.count) return;
    const int i = ta.first + threadIdx.x;
    const size_t N = b.ntot;
    T* DH = reinterpret_cast<T*>(b.dhi);
    T* DL = reinterpret_cast<T*>(b.dlo);
    T* V = reinterpret_cast<T*>(b.v);
    for (int k = 0; k < 3; ++k) {
        if (x) {
            b.x[k * N + i] = x[k * N + i];
            DH[k * N + i] = (T)0;
            if constexpr (sizeof(T) == 4) DL[k * N + i] = (T)0;
        }
        if (v) V[k * N + i] = (T)v[k * N + i];
    }
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

__device__ void force_scales(const DevSys& S, DevState& st) {
    double s_int, s_e;
    if (S.sched == SCHED_FL) { s_int = 1.0 - st.lam; s_e = st.lam; }
    else if (S.sched == SCHED_RS || S.pair >= 0) { s_int = st.lam; s_e = 0.0; }
    else if (S.sched == SCHED_NONE) { s_int = S.lam0; s_e = 0.0; }
    else { s_int = 1.0; s_e = 0.0; }
    st.scale_int = s_int;
    st.scale_E = s_e;
    st.scale_int_f = (float)s_int;
    st.scale_E_f = (float)s_e;
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
    force_scales(S, st);
    double maxrel = 0.0;
    bool scaled = false;
    for (int k = 0; k < 3; ++k) {
        const double z = st.eta[k] * dt;
        st.s[k] = (z != 0.0) ? exp(z) : 1.0;
        st.phi[k] = (z != 0.0) ? expm1(z) / z : 1.0;
        st.phi_f[k] = (float)st.phi[k];
        st.sm1_f[k] = (float)(st.s[k] - 1.0);
        scaled = scaled || (st.s[k] != 1.0);
    }
    // With no axis scaled and the cell edge still the one of the last build, the box, h = box /
    // ncell, h / hb = 1 and their FP32 copies are what they were: the FP64 divisions are skipped.
    if (scaled || st.hmoved) {
        for (int k = 0; k < 3; ++k) {
            st.box[k] *= st.s[k];
            st.h[k] = st.box[k] / (double)st.ncell[k];
            maxrel = fmax(maxrel, fabs(st.h[k] / st.hb[k] - 1.0));
        }
        refresh_box_f(st);
    }
    st.scaled = scaled ? 1 : 0;
    const double thr = 0.5 * (S.skin - maxrel * S.rcs);
    st.thr2 = thr > 0.0 ? thr * thr : -1.0;
    st.thr2_f = (float)st.thr2;
}

// carry (mode 1): the previous step's epilogue already kicked and moved the systems without a
// barostat and drew their noise for this step (k_finish with fuse): their next-step noise sums
// (ACC_XIN) become this step's (ACC_XI) and rebuild_next becomes rebuild, instead of both being
// cleared.
__global__ void __launch_bounds__(kTile) k_group(Bufs b, const DevGroup* groups, int mode, int carry) {
    const DevGroup gr = groups[blockIdx.x];
    const int members[2] = {gr.a, gr.b};
    const int nm = gr.b >= 0 ? 2 : 1;
    // The members' descriptors and states (and the pair's state) are copied into shared memory,
    // updated there by one thread (a long chain of dependent FP64 steps, each of which would
    // otherwise wait on global memory), and written back by all threads at the end.
    __shared__ __align__(16) StagedSys sh[2];
    __shared__ __align__(16) DevPair spr;
    {
        constexpr int ws = (int)(sizeof(DevSys) / 4), wt = (int)(sizeof(DevState) / 4), wp = (int)(sizeof(DevPair) / 4);
        for (int mi = 0; mi < nm; ++mi) {
            const uint32_t* gs = reinterpret_cast<const uint32_t*>(b.sys + members[mi]);
            const uint32_t* gt = reinterpret_cast<const uint32_t*>(b.st + members[mi]);
            uint32_t* ds = reinterpret_cast<uint32_t*>(&sh[mi].S);
            uint32_t* dt = reinterpret_cast<uint32_t*>(&sh[mi].st);
            for (int w = threadIdx.x; w < ws + wt; w += blockDim.x) {
                if (w < ws) ds[w] = gs[w];
                else dt[w - ws] = gt[w - ws];
            }
        }
        if (gr.pair >= 0) {
            const uint32_t* gp = reinterpret_cast<const uint32_t*>(b.pairs + gr.pair);
            uint32_t* dp = reinterpret_cast<uint32_t*>(&spr);
            for (int w = threadIdx.x; w < wp; w += blockDim.x) dp[w] = gp[w];
        }
    }
    __syncthreads();
    // decode the slot sums (fixed order: deterministic)
    if (mode != 0) {
        for (int mi = 0; mi < nm; ++mi) {
            const int s = members[mi];
            DevState& st = sh[mi].st;
            const long long* acc = b.acc + (size_t)s * ACC_N * kSlots;
            if (threadIdx.x < ACC_XI) {
                const long long sum = slot_sum(acc + (size_t)threadIdx.x * kSlots);
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
                const DevSys& S = sh[mi].S;
                DevState& st = sh[mi].st;
                if (S.pair >= 0) {
                    const DevPair& pr = spr;       // a paired system's group is its pair
                    st.lam = 1.0;
                    st.p_tgt = pr.ps;
                } else if (S.sched != SCHED_NONE) {
                    st.lam = sched_lambda(S, st.k);
                }
                force_scales(S, st);
                for (int k = 0; k < 3; ++k) {
                    st.s[k] = 1.0; st.phi[k] = 1.0; st.phi_f[k] = 1.0f; st.sm1_f[k] = 0.0f;
                }
                st.scaled = 0;
            } else {
                observe(sh[mi].S, sh[mi].st);
            }
        }
        if (mode == 1) {
            for (int mi = 0; mi < nm; ++mi) {
                const int s = members[mi];
                record_and_kick(sh[mi].S, sh[mi].st, b.dt, b.trace);
            }
            if (gr.pair >= 0) {
                DevPair& pr = spr;
                DevState& A = sh[0].st;
                DevState& B = sh[1].st;
                const DevSys& SA = sh[0].S;
                const DevSys& SB = sh[1].S;
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
                if (pr.err) { A.err |= pr.err; B.err |= pr.err; }
            } else {
                const DevSys& S = sh[0].S;
                DevState& st = sh[0].st;
                if (S.sched != SCHED_NONE) {
                    const double lam_next = sched_lambda(S, st.k + 1);
                    st.W += st.dHdl * (lam_next - st.lam);
                    st.lam = lam_next;
                }
            }
            for (int mi = 0; mi < nm; ++mi) {
                DevState& st = sh[mi].st;
                prepare_step(sh[mi].S, st, b.dt);
                st.rebuild = (carry && sh[mi].S.baro == BARO_NONE) ? st.rebuild_next : 0;
                st.rebuild_next = 0;
                st.k += 1;
            }
        }
    }
    __syncthreads();
    {
        constexpr int wt = (int)(sizeof(DevState) / 4), wp = (int)(sizeof(DevPair) / 4);
        for (int mi = 0; mi < nm; ++mi) {
            uint32_t* gt = reinterpret_cast<uint32_t*>(b.st + members[mi]);
            const uint32_t* dt = reinterpret_cast<const uint32_t*>(&sh[mi].st);
            for (int w = threadIdx.x; w < wt; w += blockDim.x) gt[w] = dt[w];
        }
        if (gr.pair >= 0) {
            uint32_t* gp = reinterpret_cast<uint32_t*>(b.pairs + gr.pair);
            const uint32_t* dp = reinterpret_cast<const uint32_t*>(&spr);
            for (int w = threadIdx.x; w < wp; w += blockDim.x) gp[w] = dp[w];
        }
    }
    // the context-wide flag word: this step's flags start from the fused epilogue's (carry) or
    // from none; the next step's word is cleared (block 0 only; no other block touches it)
    if (mode == 1 && b.any_rebuild && blockIdx.x == 0 && threadIdx.x == 0) {
        b.any_rebuild[0] = carry ? b.any_rebuild[1] : 0;
        b.any_rebuild[1] = 0;
    }
    if (mode != 2) {
        for (int mi = 0; mi < nm; ++mi) {
            long long* acc = b.acc + (size_t)members[mi] * ACC_N * kSlots;
            const bool moved = mode == 1 && carry && sh[mi].S.baro == BARO_NONE;
            for (int t = threadIdx.x; t < ACC_N * kSlots; t += blockDim.x) {
                const int a = t / kSlots;
                long long v = 0;
                if (moved && a >= ACC_XI && a < ACC_XI + 3) v = acc[t + (ACC_XIN - ACC_XI) * kSlots];
                if (a < ACC_XIN) acc[t] = v;
            }
            __syncthreads();   // ACC_XIN is read above before it is cleared
            for (int t = threadIdx.x; t < 3 * kSlots; t += blockDim.x) acc[ACC_XIN * kSlots + t] = 0;
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

__global__ void k_decode_ev(const long long* acc, double* out7) {
    const int t = threadIdx.x;
    if (t >= 7) return;
    const int a = t == 0 ? ACC_UINT : ACC_VIR + (t - 1);
    out7[t] = (double)slot_sum(acc + (size_t)a * kSlots) / kFix;
}

// ------------------------------------------------------------------------------------
// Launchers
// ------------------------------------------------------------------------------------
bool lanes_supported(int lanes) {
    return lanes == 0 || lanes == 1 || lanes == 4 || lanes == 8 || lanes == 16 || lanes == 32;
}

// With a worklist (engine) the per-tile rebuild kernels get a bounded grid and walk the
// flagged tiles; without one (stateless calls) they cover every tile.
static int rebuild_grid(const Bufs& b, int items) {
    return b.rtiles ? (items < kRebuildBlocks ? items : kRebuildBlocks) : items;
}

void launch_cells(const Bufs& b, int precision, int ntiles, int nsys, int force_all,
                  cudaStream_t s, long* launches) {
    if (ntiles <= 0) return;
    if (b.rtiles) k_rebuild_list<<<1, 256, 0, s>>>(b, nsys, force_all);
    const int g = rebuild_grid(b, ntiles);
    if (precision == NEFE_FP64) k_cells_count<double><<<g, kTile, 0, s>>>(b);
    else k_cells_count<float><<<g, kTile, 0, s>>>(b);
    k_cells_scan<<<nsys, 256, 0, s>>>(b, force_all || !b.rtiles);
    if (precision == NEFE_FP64) k_cells_fill<double><<<g, kTile, 0, s>>>(b);
    else k_cells_fill<float><<<g, kTile, 0, s>>>(b);
    // the engine's list build ranks rows by atom index and never reads perm: the in-cell order
    // (fixed by the sort for the stateless cell sort) does not matter there
    if (!b.rtiles) k_cells_sort<<<nsys, 256, 0, s>>>(b, 1);
    if (launches) *launches += 4;
}

void launch_cells_and_list(const Bufs& b, int precision, int ntiles, int nsys, int force_all,
                           cudaStream_t s, long* launches) {
    if (ntiles <= 0) return;
    launch_cells(b, precision, ntiles, nsys, force_all, s, launches);
    const int L = (b.list_lanes == 8 || b.list_lanes == 16 || b.list_lanes == 32) ? b.list_lanes : 0;
    if (L == 0) {
        const int g = b.rtiles ? kRebuildBlocks : max(1, min(kRebuildBlocks, ntiles * 8));
        if (precision == NEFE_FP64) k_nlist_cell<double><<<g, kTile, 0, s>>>(b, nsys);
        else k_nlist_cell<float><<<g, kTile, 0, s>>>(b, nsys);
        if (launches) *launches += 1;
        return;
    }
    const int g = rebuild_grid(b, ntiles * L);
    if (precision == NEFE_FP64) {
        if (L == 8) k_nlist<double, 8><<<g, kTile, 0, s>>>(b);
        else if (L == 16) k_nlist<double, 16><<<g, kTile, 0, s>>>(b);
        else k_nlist<double, 32><<<g, kTile, 0, s>>>(b);
    } else {
        if (L == 8) k_nlist<float, 8><<<g, kTile, 0, s>>>(b);
        else if (L == 16) k_nlist<float, 16><<<g, kTile, 0, s>>>(b);
        else k_nlist<float, 32><<<g, kTile, 0, s>>>(b);
    }
    if (launches) *launches += 1;
}

int rebuild_coop_blocks(int precision) {
    int per_sm = 0, dev = 0, sms = 0;
    cudaError_t e = precision == NEFE_FP64
                        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rebuild_coop<double>, kTile, 0)
                        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rebuild_coop<float>, kTile, 0);
    if (e != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return min(per_sm * sms, kRebuildBlocks);
}

void launch_rebuild_coop(const Bufs& b, int precision, int blocks, int nsys, cudaStream_t s, long* launches) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)blocks);
    cfg.blockDim = dim3(kTile);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;   // every block resident: the grid barriers can complete
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if (precision == NEFE_FP64) cudaLaunchKernelEx(&cfg, k_rebuild_coop<double>, b, nsys);
    else cudaLaunchKernelEx(&cfg, k_rebuild_coop<float>, b, nsys);
    if (launches) *launches += 1;
}

int check_barrier_timeout(double limit_ms) {
    void* p = nullptr;
    if (cudaMalloc(&p, 2 * sizeof(int)) != cudaSuccess) return -2;
    cudaMemset(p, 0, 2 * sizeof(int));
    unsigned* word = static_cast<unsigned*>(p);
    int* tmo = static_cast<int*>(p) + 1;
    k_barrier_selftest<<<4, kTile>>>(word, tmo, (unsigned long long)(limit_ms * 1e6));
    int h = 0;
    const cudaError_t e = cudaMemcpy(&h, tmo, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(p);
    if (e != cudaSuccess) return -3;
    return h ? 1 : 0;
}

void launch_aos_soa(const double* src, double* dst, int n, int to_soa, cudaStream_t s) {
    if (n <= 0) return;
    const int blocks = (3 * n + 255) / 256;
    if (to_soa) k_aos_to_soa<<<blocks, 256, 0, s>>>(src, dst, n);
    else k_soa_to_aos<<<blocks, 256, 0, s>>>(src, dst, n);
}

__global__ void k_decode_grad(const long long* acc, double* out8) {
    const int t = threadIdx.x;
    if (t >= 8) return;
    const int a = t == 0 ? ACC_UINT : ACC_DTH + (t - 1);
    out8[t] = (double)slot_sum(acc + (size_t)a * kSlots) / kFix;
}

void launch_decode_grad(const long long* acc, double* out8, cudaStream_t s) {
    k_decode_grad<<<1, 32, 0, s>>>(acc, out8);
}

void launch_decode_ev(const long long* acc, double* out7, cudaStream_t s) {
    k_decode_ev<<<1, 32, 0, s>>>(acc, out7);
}

void launch_uf_list(const Bufs& b, int precision, int ntiles, cudaStream_t s, long* launches) {
    if (ntiles <= 0 || !b.uf_nbr) return;
    const int g = rebuild_grid(b, ntiles);
    if (precision == NEFE_FP64) k_uflist<double><<<g, kTile, 0, s>>>(b);
    else k_uflist<float><<<g, kTile, 0, s>>>(b);
    if (launches) *launches += 1;
}

void launch_uf(const Bufs& b, int precision, int ntiles, int mode, cudaStream_t s, long* launches) {
    if (ntiles <= 0 || !b.uf_nbr) return;
    if (precision == NEFE_FP64) {
        if (mode == FM_FORCES) k_uf<double, FM_FORCES><<<ntiles, kTile, 0, s>>>(b);
        else k_uf<double, FM_STEP><<<ntiles, kTile, 0, s>>>(b);
    } else {
        if (mode == FM_FORCES) k_uf<float, FM_FORCES><<<ntiles, kTile, 0, s>>>(b);
        else k_uf<float, FM_STEP><<<ntiles, kTile, 0, s>>>(b);
    }
    if (launches) *launches += 1;
}

void launch_kick_drift(const Bufs& b, int precision, int ntiles, int mode, cudaStream_t s, long* launches,
                       int skip) {
    if (ntiles <= 0) return;
    if (precision == NEFE_FP64) k_kick_drift<double><<<ntiles, kTile, 0, s>>>(b, mode, skip);
    else k_kick_drift<float><<<ntiles, kTile, 0, s>>>(b, mode, skip);
    if (launches) *launches += 1;
}

void launch_mirror(const Bufs& b, int precision, int ntiles, cudaStream_t s, long* launches) {
    if (ntiles <= 0) return;
    if (precision == NEFE_FP64) k_mirror<double><<<ntiles, kTile, 0, s>>>(b);
    else k_mirror<float><<<ntiles, kTile, 0, s>>>(b);
    if (launches) *launches += 1;
}

template <typename T>
static void edges_dispatch(const Bufs& b, int lanes, int ntiles, cudaStream_t s) {
    // an FP64 shell of 32 atoms per block does not fit the 48 KB static shared limit: 4 -> 8
    switch (lanes) {
        case 0:   // one thread per atom, scatter form: FP32 only
        case 1: { // one thread per atom: FP32 only (the FP64 columns exceed the shared limit)
            if constexpr (sizeof(T) == 8) {
                k_edges<T, 8><<<ntiles * 8, kTile, 0, s>>>(b);
            } else {
                const int items = ntiles * (kTile / kEdges1Threads);
                if (lanes == 0) k_edges1<T, true><<<items, kEdges1Threads, 0, s>>>(b);
                else k_edges1<T, false><<<items, kEdges1Threads, 0, s>>>(b);
            }
            break;
        }
        case 4:
            if constexpr (sizeof(T) == 8) k_edges<T, 8><<<ntiles * 8, kTile, 0, s>>>(b);
            else k_edges<T, 4><<<ntiles * 4, kTile, 0, s>>>(b);
            break;
        case 8: k_edges<T, 8><<<ntiles * 8, kTile, 0, s>>>(b); break;
        case 16: k_edges<T, 16><<<ntiles * 16, kTile, 0, s>>>(b); break;
        default: k_edges<T, 32><<<ntiles * 32, kTile, 0, s>>>(b); break;
    }
}

void launch_edges(const Bufs& b, int precision, int lanes, int ntiles, int mode, cudaStream_t s,
                  long* launches) {
    (void)mode;
    if (ntiles <= 0) return;
    if (precision == NEFE_FP64) edges_dispatch<double>(b, lanes, ntiles, s);
    else edges_dispatch<float>(b, lanes, ntiles, s);
    if (launches) *launches += 1;
}

template <typename T, int MODE>
static void gather_dispatch(const Bufs& b, int lanes, int ntiles, cudaStream_t s, int fuse) {
    switch (lanes) {
        case 0: k_finish<T, MODE><<<ntiles, kTile, 0, s>>>(b, fuse); break;
        case 1: k_gather<T, MODE, 1><<<ntiles, kTile, 0, s>>>(b); break;
        case 2: k_gather<T, MODE, 2><<<ntiles * 2, kTile, 0, s>>>(b); break;
        case 8: k_gather<T, MODE, 8><<<ntiles * 8, kTile, 0, s>>>(b); break;
        default: k_gather<T, MODE, 4><<<ntiles * 4, kTile, 0, s>>>(b); break;
    }
}

void launch_gather(const Bufs& b, int precision, int lanes, int ntiles, int mode, cudaStream_t s,
                   long* launches, int fuse) {
    if (ntiles <= 0) return;
    if (precision == NEFE_FP64) {
        if (mode == FM_FORCES) gather_dispatch<double, FM_FORCES>(b, lanes, ntiles, s, 0);
        else if (mode == FM_SETUP) gather_dispatch<double, FM_SETUP>(b, lanes, ntiles, s, 0);
        else gather_dispatch<double, FM_STEP>(b, lanes, ntiles, s, fuse);
    } else {
        if (mode == FM_FORCES) gather_dispatch<float, FM_FORCES>(b, lanes, ntiles, s, 0);
        else if (mode == FM_SETUP) gather_dispatch<float, FM_SETUP>(b, lanes, ntiles, s, 0);
        else gather_dispatch<float, FM_STEP>(b, lanes, ntiles, s, fuse);
    }
    if (launches) *launches += 1;
}

void launch_materialize(const Bufs& b, int precision, int ntiles, double* x, double* v, cudaStream_t s) {
    if (ntiles <= 0) return;
    if (precision == NEFE_FP64) k_materialize<double><<<ntiles, kTile, 0, s>>>(b, x, v);
    else k_materialize<float><<<ntiles, kTile, 0, s>>>(b, x, v);
}

void launch_inject(const Bufs& b, int precision, int ntiles, const double* x, const double* v, cudaStream_t s) {
    if (ntiles <= 0) return;
    if (precision == NEFE_FP64) k_inject<double><<<ntiles, kTile, 0, s>>>(b, x, v);
    else k_inject<float><<<ntiles, kTile, 0, s>>>(b, x, v);
}

void launch_group(const Bufs& b, const DevGroup* groups, int ngroups, int mode, cudaStream_t s,
                  long* launches, int carry) {
    if (ngroups <= 0) return;
    k_group<<<ngroups, kTile, 0, s>>>(b, groups, mode, carry);
    if (launches) *launches += 1;
}

void launch_noise(unsigned long long seed, unsigned long long sys_id, unsigned long long step, int n,
                  int precision, double* xi, cudaStream_t s) {
    if (n <= 0) return;
    k_noise<<<(n + 127) / 128, 128, 0, s>>>(seed, sys_id, step, n, precision, xi);
}

}  // namespace nefe
