// Host-side launchers of the libnefe kernels (defined in nefe_kernels.cu).
#pragma once
#include <cuda_runtime.h>
#include "nefe_dev.h"

namespace nefe {

constexpr int kSlots = 32;   // accumulator slots per system (spreads atomics over 32 words)

// Pointers handed to every kernel.  Per-atom arrays are global over all systems of a
// context; FP64 SoA arrays have stride ntot.  F/xs/xsb are float4 (FP32 path) or double4.
struct Bufs {
    const DevSys* sys;
    DevState* st;
    long long* acc;          // [nsys][ACC_N][kSlots]
    const int* tile_sys;     // system of each 128-atom tile
    double* x;               // FP64 anchor positions (positions at the last list build), SoA
    void* dhi;               // displacement since the last build, kernel precision, SoA (may be NULL)
    void* dlo;               // its compensation term (FP32 path; may be NULL)
    void* v;                 // velocities, kernel precision, SoA
    const double* r0;        // Einstein sites, FP64 SoA
    void* F;                 // total force used by the next half kick (T4)
    void* xs;                // mirror x - q h (T4)
    void* xa;                // mirror at the last build (T4)
    void* xcs;               // mirror at the last build in cell order, atom index in .w (T4)
    void* sd0;               // anchor - r0 at the last build (T4)
    void* xi;                // thermostat noise of the current step (T4)
    void* shd;               // [ntot][kShell] in-cutoff shell: d_ij and g_ij (T4)
    int* shj;                // [ntot][kShell] shell neighbour indices
    int* shn;                // shell size
    void* spill;             // thread-per-atom pass A: shell entries beyond its shared table, or NULL
    void* P;                 // [ntot] pass-A force (.w = atom energy), then [ntot][2] its virial (T4)
    int4* q;                 // unwrapped cell index per axis, from the last build
    int* cell_of;
    int* perm;
    int* cell_start;         // per system: ncell_cap + 1 entries at cell0 + system index
    int* cell_count;
    int* cell_cursor;
    int* nbr;
    int* cnt;
    int cap;
    int nbr_il;              // 0: rows row-major (entry k of atom i at i cap + k); 1 (engine, cap a
                             // multiple of 4): interleaved by 4 -- entries 4g..4g+3 of every atom
                             // form one 16-byte vector, the vectors of consecutive atoms adjacent
                             // (at (g ntot + i) 4 + k % 4), and each row is padded to a multiple
                             // of 4 with entries that never pass the distance test
    int ntot;
    int tile_base;           // first tile of the launch (force passes run in L2-sized chunks)
    int* rtiles;             // rebuild worklist (tiles of flagged systems) or NULL
    int* rcount;             // its length
    int* rcbase;             // [nsys + 1] first worklist cell of each system (cells of flagged
                             // systems, in system order; the last entry is their number) or NULL
    double dt;
    const void* swc;         // SWc<float> or SWc<double> table
    DevPair* pairs;
    double* trace;
    double* f_out;           // stateless: FP64 SoA forces
    double* e_atom;          // stateless: per-atom energy (may be NULL)
    int want_grad;           // pass A also sums dE/d(A, B, p, q, a, lambda3, gamma)
    int list_lanes;          // list build: 0 one warp per cell; 8, 16 or 32 lanes per atom
    int* uf_nbr;             // [ntot][kUfCap] Uhlenbeck-Ford pair rows (NULL: no UF system)
    int* uf_cnt;             // [ntot] their lengths
    void* uf_F;              // [ntot] UF force and atom energy of the step (T4)
    const int* uf_tiles;     // tiles of the UF systems (per-step UF kernel), or NULL: every tile
    int* lacc;               // [ntot][4] int32 force accumulators of the scatter form (2^-21 eV/A)
    int* any_rebuild;        // engine: [0] some system's rebuild flag is set this step, [1] some
                             // rebuild_next is set (fused epilogue); NULL in the stateless calls
    int rebuild_all;         // engine: when any system's list is stale, every system rebuilds (one
                             // full-width build instead of many narrow ones)
};

enum ForceMode { FM_FORCES = 0, FM_SETUP = 1, FM_STEP = 2 };

// Cell count / scan / fill / sort only (the stateless cell sort).
void launch_cells(const Bufs& b, int precision, int ntiles, int nsys, int force_all,
                  cudaStream_t s, long* launches);
// Decodes one system's fixed-point sums into [U_int, virial xx yy zz xy xz yz] (FP64, device).
void launch_decode_ev(const long long* acc, double* out7, cudaStream_t s);
// Decodes [U_int, dE/dA, dE/dB, dE/dp, dE/dq, dE/da, dE/dlambda3, dE/dgamma] (FP64, device).
void launch_decode_grad(const long long* acc, double* out8, cudaStream_t s);
// Rebuild sequence (only systems whose rebuild flag is set, or all when force_all).
void launch_cells_and_list(const Bufs& b, int precision, int ntiles, int nsys, int force_all,
                           cudaStream_t s, long* launches);
// Half kick + drift + mirror + displacement check + noise sums (mode 0: no kick/drift).  skip:
// the systems without a barostat were moved by the previous step's fused epilogue.
void launch_kick_drift(const Bufs& b, int precision, int ntiles, int mode, cudaStream_t s,
                       long* launches, int skip = 0);
// Uhlenbeck-Ford pair rows of the UF systems (after the cell fill; flagged systems only when a
// rebuild worklist is set).
void launch_uf_list(const Bufs& b, int precision, int ntiles, cudaStream_t s, long* launches);
// Uhlenbeck-Ford forces and energies over `ntiles` tiles (b.uf_tiles, or every tile when NULL);
// mode FM_FORCES writes b.f_out / b.e_atom (stateless), otherwise b.uf_F for pass B.
void launch_uf(const Bufs& b, int precision, int ntiles, int mode, cudaStream_t s, long* launches);
// Force pass A (edges: pair terms, triplets centred on each atom, leg forces per edge).
void launch_edges(const Bufs& b, int precision, int lanes, int ntiles, int mode, cudaStream_t s,
                  long* launches);
// Force pass B (gather leg forces; springs, Langevin and second half kick in FM_SETUP/FM_STEP).
// fuse (scatter form, FM_STEP): systems without a barostat go on to the next step's kick, drift
// and noise in the same kernel.
void launch_gather(const Bufs& b, int precision, int lanes, int ntiles, int mode, cudaStream_t s,
                   long* launches, int fuse = 0);
// FP64 positions (anchor + displacement) and FP64 velocities into SoA staging buffers.
void launch_materialize(const Bufs& b, int precision, int ntiles, double* x, double* v, cudaStream_t s);
// Replace positions (anchor, zero displacement) and/or velocities from FP64 SoA buffers.
void launch_inject(const Bufs& b, int precision, int ntiles, const double* x, const double* v, cudaStream_t s);
// Per-group scalar update. mode 0 INIT, 1 STEP, 2 OBSERVE.  carry (STEP): the previous epilogue
// was fused (its next-step noise sums and rebuild flag are moved into place).
void launch_group(const Bufs& b, const DevGroup* groups, int ngroups, int mode, cudaStream_t s,
                  long* launches, int carry = 0);
// Mirror only (stateless force entry): q and xs from x with the list-build formula.
void launch_mirror(const Bufs& b, int precision, int ntiles, cudaStream_t s, long* launches);
// Thermostat noise as FP64 (n,3).
void launch_noise(unsigned long long seed, unsigned long long sys_id, unsigned long long step,
                  int n, int precision, double* xi, cudaStream_t s);

// The engine's single-launch rebuild (cooperative; see k_rebuild_coop): the largest grid whose
// blocks are all resident (0 if it cannot be launched), and its launch.
int rebuild_coop_blocks(int precision);
void launch_rebuild_coop(const Bufs& b, int precision, int blocks, int nsys, cudaStream_t s, long* launches);
// Runs the barrier time-limit check on the current device: 1 timed out (expected), 0 did not,
// negative on a CUDA error.
int check_barrier_timeout(double limit_ms);

bool lanes_supported(int lanes);
// (n,3) row-major <-> SoA (to_soa = 1: aos -> soa).
void launch_aos_soa(const double* src, double* dst, int n, int to_soa, cudaStream_t s);

}  // namespace nefe
