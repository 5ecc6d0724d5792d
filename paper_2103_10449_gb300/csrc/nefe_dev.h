// Internal layout of libnefe: device-side descriptors shared by the kernels and the host
// engine.  Plain structs only (no CUDA types), so host code includes it freely.
#pragma once
#include <stdint.h>

namespace nefe {

// Metal units.  kB and hbar are CODATA 2018; MVV2E converts (g/mol) A^2/ps^2 to eV.
constexpr double kB = 8.617333262e-5;
constexpr double kMvv2e = 1.66053906660e-23 / 1.602176634e-19;
constexpr double kEvA3ToGPa = 160.21766340;   // 1 eV/A^3 in GPa (1.602176634e-19 J / 1e-30 m^3)

constexpr int kTile = 128;        // atoms per tile; a tile never straddles two systems
constexpr int kShell = 32;        // max neighbours inside a*sigma held per atom
constexpr int kSpill1 = 12;       // thread-per-atom pass A: shell entries kept in global memory
constexpr int kMaxCap = 64;       // max neighbour row capacity (one 64-bit slot mask per atom)
constexpr int kCodeShift = 27;    // nbr entry = j | (cell-offset code << 27)
constexpr uint32_t kIndexMask = (1u << kCodeShift) - 1u;
// Uhlenbeck-Ford pair list: entry = j | (code << 25), code = (ox+2) + 5 (oy+2) + 25 (oz+2) for the
// cell offset o in {-2..2}^3 through which j was reached.
constexpr int kUfCap = 256;
constexpr int kUfShift = 25;
constexpr uint32_t kUfMask = (1u << kUfShift) - 1u;

// Fixed-point accumulators: per-system sums are accumulated as int64 in units of 2^-32,
// so the order in which blocks add them does not change the result (bitwise determinism).
constexpr double kFix = 4294967296.0;
enum Acc {
    ACC_UINT = 0,       // U_int (unscaled SW, or Einstein test potential)
    ACC_UREF,           // U_E (FL reference)
    ACC_VIR,            // 6: SW virial xx yy zz xy xz yz (unscaled)
    ACC_KT = ACC_VIR + 6,   // 6: sum m v_a v_b (eV)
    ACC_XI = ACC_KT + 6,    // 3: sum of thermostat normals of the current step
    ACC_DTH = ACC_XI + 3,   // 7: dE/d(A, B, p, q, a, lambda3, gamma) (stateless gradient call)
    ACC_XIN = ACC_DTH + 7,  // 3: sum of the next step's thermostat normals, drawn by an epilogue
                            //    that already moved the atoms (becomes ACC_XI at the next step)
    ACC_N = ACC_XIN + 3
};

enum Sched { SCHED_NONE = 0, SCHED_FL = 1, SCHED_RS = 2, SCHED_AS = 3 };
enum Pot { POT_SW = 0, POT_EINSTEIN = 1, POT_UF = 2 };
enum UfMode { UF_NONE = 0, UF_INT = 1, UF_REF = 2 };   // UF as U_int, or as the FL reference
enum Baro { BARO_NONE = 0, BARO_ISO = 1, BARO_ANISO = 2 };

// Potential constants in the precision of the force kernel.
template <typename T>
struct SWc {
    T inv_sig;     // 1/sigma
    T a;           // cutoff in sigma units
    T rc2;         // (a sigma)^2
    T epsA;        // eps * A
    T B, p, q;
    T epslam;      // eps * lambda3
    T gam;
    T c0;
    T eps, A, lam3;  // for the parameter derivatives
    T s_act;       // edges with r/sigma >= s_act are dropped (see make_swc)
    T act2;        // (s_act sigma)^2
    int int_pq;    // 1 when p == 4 and q == 0 (the standard set): s^-p by multiplications
};

// Per-system description (constant during a run).
struct DevSys {
    int off, n;                 // first atom, atom count
    int tile0, ntile;           // first tile, tile count
    int cell0, ncell_cap;       // first cell slot, cell capacity (cell_start uses +1 per system)
    int pot, sched, direction, baro;
    long long nsched;
    double k_int, k_E, lam_f, p_phys, p0, p1, lam0;   // pressures in eV/A^3
    double mass_e;              // mass * MVV2E (eV ps^2 / A^2)
    double T, tdamp;
    unsigned long long seed;
    int rng_id;                 // system index fed to the noise counter
    int pair;                   // dCCI pair index or -1
    double p_ext, pdamp;        // barostat target for SCHED_NONE (eV/A^3), damping (ps)
    double rcs, skin;           // list radius and skin (A)
    double amp;                 // Langevin noise amplitude sqrt(2 m kB T / (tdamp dt)) (eV/A)
    double gam;                 // Langevin friction m / tdamp (eV ps / A^2)
    double ckick;               // dt / (2 m) (A^2 / (eV ps))
    // FP32 copies and flags read by the FP32 kernels (no FP64 instruction per atom)
    float amp_f, gam_f, ckick_f, mass_f, kE_f, kint_f, dt_f, inv_n_f;
    float rcs2_lo_f, rcs2_hi_f; // list radius^2 times (1 -/+ 1e-4): FP32 filter band
    int thermo;                 // tdamp > 0
    int springs;                // an Einstein spring acts (FL reference or U_int = Einstein)
    int trace_every;
    long long trace_cap, trace_off;
    int prm;                    // index into the parameter tables
    // Uhlenbeck-Ford term: u = -pk ln(1 - exp(-r^2 is2)) - shift for r^2 < rc2
    int uf_mode;                // UfMode
    double uf_pk, uf_is2, uf_rc2, uf_shift, uf_R2;   // p kB T (eV), 1/sigma^2, rc^2, u(rc), list radius^2
    float uf_pk_f, uf_is2_f, uf_rc2_f, uf_shift_f, uf_R2_f;
};

// Per-system dynamic state.
struct DevState {
    double box[3];
    double h[3];                // cell edge at the current box: box / ncell
    double hb[3];               // cell edge at the last list build
    int ncell[3];
    int rebuild;                // set by any atom that moved too far; cleared each step
    double eta[3];              // barostat strain rates (1/ps)
    double lam, W, p_tgt;
    long long k;                // steps completed
    double u_int, u_ref, vir[6], kt[6];
    double sums[5];             // running sums: H, dH/dl, P, V, count
    double s[3], phi[3];        // drift factors for the current step
    double scale_int, scale_E;  // force scales at the current lambda
    double thr2;                // squared displacement that triggers a rebuild
    double dHdl, H, V, P[6];    // last observation
    unsigned err;
    int rebuild_next;           // set by the epilogue that already moved the atoms for the next
                                // step (systems without a barostat); becomes `rebuild` at that step
    long long trace_n;
    long long nbuild;           // list builds so far
    // FP32 copies of this step's constants (written with their FP64 sources)
    float h_f[3], hb_f[3], rho_f[3], phi_f[3], sm1_f[3];
    float scale_int_f, scale_E_f, thr2_f;
    int scaled;                 // s != 1 on some axis (barostat moved the box this step)
    int hmoved;                 // h != hb on some axis (box differs from the last build)
    double ibox[3];             // 1 / box at the last list build (set with the grid by k_rebuild_list)
    double gbox[3], grcs;       // box and list radius the cell grid was computed for (0: never)
};

struct DevPair {
    int a, b, mode, pad;
    double T0, frm, to;         // TEMP: K; PRESS: eV/A^3
    long long nsteps, k;
    double lam, ps;             // current lambda and scaled pressure (eV/A^3)
    unsigned err;
    int pad2;
};

// One group per independent update unit: a single system (b = -1) or a dCCI pair.
struct DevGroup {
    int a, b, pair, pad;
};

}  // namespace nefe
