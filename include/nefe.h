/*
 * nefe.h - C ABI of libnefe.so: GB300 (sm_103a) kernels for non-equilibrium free-energy
 * and dynamic Clausius-Clapeyron integration (dCCI) runs of Stillinger-Weber silicon.
 *
 * The operations are those of Cajahuaringa & Antonelli, "Non-equilibrium free-energy
 * calculation of phase-boundaries using LAMMPS" (arXiv:2103.10449):
 *   - adiabatic switching and its dynamical work (Sec. 2, Eq. Wdyn), accumulated left-point;
 *   - Hamiltonian interpolation to an Einstein crystal (Sec. 2.1, Eqs. H_lambda, Wrev_HI, dA);
 *   - reversible scaling in NPT (Sec. 2.2, Eqs. H_RS, T_sc, P_sc, dH_RS);
 *   - adiabatic switching in pressure (Sec. 2.3, Eqs. Wmech, Wmech_dyn);
 *   - the discrete dCCI updates (Sec. 3, Eqs. Ps_coex_discreted and l_coex_discreted);
 *   - velocity-Verlet + Langevin thermostat ("zero yes") + a Parrinello-Rahman-type box
 *     equation whose target pressure is multiplied by lambda (Sec. 4, the "ners" tag);
 *   - the Stillinger-Weber potential of Sec. 4 (functional form of Stillinger & Weber 1985).
 *
 * Conventions shared by every call:
 *   - Every call returns int: NEFE_OK (0) or a negative NEFE_E* code.  No call aborts,
 *     throws or prints.  nefe_last_error() returns a static, NUL-terminated message for the
 *     most recent failure on the calling thread.
 *   - Units are LAMMPS "metal": Angstrom, eV, ps, g/mol, K.  Pressures cross the ABI in GPa.
 *   - "device" pointers are CUDA device memory on the context's / call's device, owned by
 *     the caller unless stated otherwise; "host" pointers are ordinary host memory.
 *   - Device FP64 positions are structure-of-arrays: x[0..n) = x, x[n..2n) = y,
 *     x[2n..3n) = z.  Host positions, velocities and forces are (n, 3) row-major.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).  Calls
 *     are asynchronous on it unless documented as blocking.
 */
#ifndef NEFE_H
#define NEFE_H

#include <stdint.h>

#if defined(__GNUC__)
#define NEFE_API __attribute__((visibility("default")))
#else
#define NEFE_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status codes */
#define NEFE_OK         0
#define NEFE_EINVAL    -1   /* bad argument (NULL pointer, n < 0, box too small, ...)  */
#define NEFE_ENOMEM    -2   /* a device or host allocation failed                       */
#define NEFE_ECUDA     -3   /* a CUDA runtime call failed                               */
#define NEFE_EOVERFLOW -4   /* a neighbour row or an in-cutoff shell exceeded capacity  */
#define NEFE_ENAN      -6   /* non-finite energy, force or pressure                     */
#define NEFE_EDEGEN    -7   /* dCCI: |dV| (temperature control) or |dU| (pressure       */
                            /* control) per atom fell below the singularity guard       */
#define NEFE_ETIMEOUT  -8   /* a bounded device wait gave up                            */
#define NEFE_ESTATE    -9   /* call not valid in the context's current state            */

/* Per-system error word bits (nefe_results.error). */
#define NEFE_ERR_NBR_OVERFLOW   0x1u   /* neighbour row longer than the row capacity     */
#define NEFE_ERR_SHELL_OVERFLOW 0x2u   /* more than 32 neighbours inside a*sigma         */
#define NEFE_ERR_NAN            0x4u   /* non-finite energy or pressure                  */
#define NEFE_ERR_DEGEN          0x8u   /* dCCI singular update (see NEFE_EDEGEN)         */
#define NEFE_ERR_BOX            0x10u  /* box below 2 (rc + skin) or cell grid too large */
#define NEFE_ERR_CELL           0x20u  /* cell occupancy inconsistent with the atom count   */
#define NEFE_ERR_TIMEOUT        0x40u  /* a grid barrier of the list rebuild gave up waiting */

/* Precision of the force kernel.  Positions, box, energies, virial and work are FP64 in
 * both; NEFE_FP32 evaluates the pair and triplet arithmetic in FP32.                   */
#define NEFE_FP32 0
#define NEFE_FP64 1

/* ---------------------------------------------------------------- potential */
/* Stillinger-Weber parameters (Stillinger & Weber 1985; the paper's Sec. 4 uses the
 * standard silicon set: eps 2.1683 eV, sigma 2.0951 A, A 7.049556277, B 0.6022245584,
 * p 4, q 0, a 1.80, lambda3 21.0, gamma 1.20, cos0 -1/3).
 *   E = sum_{i<j} eps A (B s^-p - s^-q) exp(1/(s - a))                  (s = r/sigma < a)
 *     + sum_i sum_{j<k} eps lambda3 (cos theta_jik - cos0)^2
 *                       exp(gamma/(s_ij - a)) exp(gamma/(s_ik - a))                     */
typedef struct nefe_sw_params {
    double eps, sigma, A, B, p, q, a, lambda3, gamma, cos0;
} nefe_sw_params;

/* Fills *out with the standard silicon set above.  Never fails for a non-NULL out. */
NEFE_API int nefe_sw_params_silicon(nefe_sw_params* out);

/* Reference system of the Hamiltonian interpolation (NEFE_SCHED_FL, Sec. 2.1): the Einstein
 * crystal for solids, the Uhlenbeck-Ford fluid for liquids. */
#define NEFE_REF_EINSTEIN 0
#define NEFE_REF_UF       1

/* Uhlenbeck-Ford fluid (Sec. 2.1 names it the fluid-phase reference, Paula Leite et al. 2016;
 * Sec. 4 uses p = 25, sigma = 2.0 for liquid Si at 2200 K):
 *   u(r) = -p kB T ln(1 - exp(-r^2/sigma^2)) - u(rc)  for r < rc, else 0,
 * truncated at rc and shifted so that the energy is continuous there.  T is the reference's
 * own temperature (it sets the energy scale p kB T; it need not equal the thermostat's).
 * The pair list radius is rc + skin and must not exceed 2 (a sigma + skin) (the cells of the
 * SW list are reused with a +-2 cell stencil); rows hold at most NEFE_UF_CAP neighbours.    */
typedef struct nefe_uf_params {
    double p, sigma, T, rc;
} nefe_uf_params;
#define NEFE_UF_CAP 256

/* ---------------------------------------------------------------- stateless kernels */
/*
 * nefe_cell_bin - cell grid, cell of each atom and the stable counting sort by cell.
 * Defines the cell list the neighbour search walks (not printed in the paper; LAMMPS
 * builds it implicitly, Plimpton 1995).
 *   x           device, FP64 SoA [3n], unwrapped coordinates.
 *   n           atoms (n >= 0; n == 0 is a no-op that still reports the grid).
 *   box         host [3], orthorhombic box lengths; each must give >= 2 cells.
 *   rcs         cell criterion: per axis ncell = floor(L/rcs), reduced by one while
 *               L/ncell < rcs (1 + 1e-9).
 *   ncell3      host out [3], cells per axis.
 *   cell_of     device out [n], cell id cx + nx (cy + ny cz) with c = (int)(w ncell),
 *               w = x/L - floor(x/L).
 *   cell_start  device out [ncell_cap + 1]; entries 0..ncells hold the exclusive prefix
 *               sum of the cell occupancy.
 *   perm        device out [n], atom indices ordered by (cell id, atom index).
 *   ncell_cap   capacity of cell_start minus one.
 * Scratch: one int per cell, allocated stream-ordered on `stream` and released before
 * return of the stream work.  Returns NEFE_EINVAL on bad arguments or too few / too many
 * cells, NEFE_ENOMEM when the scratch allocation fails.  Blocking: no.
 */
NEFE_API int nefe_cell_bin(const double* x, int n, const double box[3], double rcs,
                  int ncell3[3], int* cell_of, int* cell_start, int* perm, int ncell_cap,
                  void* stream);

/*
 * nefe_cell_bin_noalloc - the same cell grid, cell ids, occupancy prefix sum and stable sort
 * as nefe_cell_bin (identical outputs for identical inputs), for callers that cannot allocate
 * device memory: code running under another framework's memory pool, real-time loops that
 * must never enter the CUDA allocator, or processes whose device memory is reserved up
 * front.  It calls no cudaMalloc, cudaFree, cudaMallocAsync or allocating library routine.
 * (The paper has no counterpart: this is a deployment variant of the cell sort.)
 *   Arguments and outputs as nefe_cell_bin; the caller still owns x, cell_of, cell_start
 *   and perm.
 *   Limits: n <= NEFE_NOALLOC_MAX_ATOMS and at most NEFE_NOALLOC_MAX_CELLS cells; larger
 *   inputs return NEFE_EINVAL with a message naming the limit.
 *   Scratch: one fixed __device__ array of about 3.6 MB in libnefe.so, held on every GPU
 *   that loads the library until the process exits.  Every call shares it and it keeps the
 *   previous call's contents (the occupancy counts are cleared by each call), so calls
 *   whose GPU work may overlap (different streams, or different host threads on the same
 *   device) race and must be serialised by the caller.  The first call on a device looks up
 *   the array's device address (cudaGetSymbolAddress) with that device current; make that
 *   first call before any stream capture.  Blocking: no.
 */
#define NEFE_NOALLOC_MAX_ATOMS 65536
#define NEFE_NOALLOC_MAX_CELLS 65536
NEFE_API int nefe_cell_bin_noalloc(const double* x, int n, const double box[3], double rcs,
                                   int ncell3[3], int* cell_of, int* cell_start, int* perm,
                                   int ncell_cap, void* stream);

/*
 * nefe_neighbor_build - Verlet list with skin: for each i every j != i with minimum-image
 * d = x_j - x_i - m L, (d_x^2 + d_y^2) + d_z^2 < rcs^2 decided in FP64 (strict <), rows
 * ordered by ascending j.  (The paper relies on LAMMPS's list, Plimpton 1995; this is its
 * plain definition.)
 *   x, n, box   as nefe_cell_bin; every box length must be >= 2 rcs.
 *   rcs         list radius rc + skin (A).
 *   cap         row capacity (1..64).
 *   nbr         device out [n * cap] int32; entry = j | (code << 27) where
 *               code = (ox+1) + 3 (oy+1) + 9 (oz+1) is the cell offset o in {-1,0,1}^3
 *               through which j was reached: d = (x_j - q_j h) - (x_i - q_i h) + o h with
 *               q = floor(x/L) ncell + c the unwrapped cell index and h = L/ncell.
 *   cnt         device out [n], true row lengths (may exceed cap: overflow).
 *   overflow    host out, 1 if some row exceeded cap (rows are then truncated), else 0.
 *               Reading it synchronises `stream`.
 * Returns NEFE_EINVAL for bad arguments, NEFE_ENOMEM/NEFE_ECUDA on runtime failure,
 * NEFE_EOVERFLOW when a row exceeded cap.  Blocking: yes (reads the overflow flag).
 */
NEFE_API int nefe_neighbor_build(const double* x, int n, const double box[3], double rcs, int cap,
                        int* nbr, int* cnt, int* overflow, void* stream);

/*
 * nefe_sw_forces - Stillinger-Weber energy, forces and virial on a list built by
 * nefe_neighbor_build from the same x and box.  Gather formulation: the force on i sums the
 * pair terms, the three-body terms centred on i, and the three-body terms centred on each
 * neighbour j in which i is a leg, so no atomics touch the forces and the result is
 * bitwise reproducible.
 *   x, n, box, rcs, nbr, cnt, cap   as nefe_neighbor_build (same values).
 *   prm         host, potential parameters (prm->a * prm->sigma <= rcs).
 *   precision   NEFE_FP32 or NEFE_FP64 pair/triplet arithmetic.
 *   f           device out, FP64 SoA [3n] forces (eV/A).
 *   e_atom      device out [n] or NULL: per-atom energy (half of each pair term, each
 *               three-body term to its centre atom).
 *   energy_virial device out [7] or NULL: total energy then the virial W_ab =
 *               sum over terms of sum_legs (x_leg - x_centre)_a f_leg_b as
 *               xx, yy, zz, xy, xz, yz (eV), each summed in FP64.
 *   shell_overflow host out or NULL: 1 if some atom had more than 32 neighbours inside
 *               a*sigma (their forces are then incomplete).  Reading it synchronises.
 * Returns NEFE_EINVAL, NEFE_ENOMEM, NEFE_ECUDA or NEFE_EOVERFLOW (shell overflow).
 */
NEFE_API int nefe_sw_forces(const double* x, int n, const double box[3], double rcs,
                   const int* nbr, const int* cnt, int cap, const nefe_sw_params* prm,
                   int precision, double* f, double* e_atom, double* energy_virial,
                   int* shell_overflow, void* stream);

/*
 * nefe_uf_forces - Uhlenbeck-Ford energy, forces and virial (the fluid reference of Sec. 2.1;
 * functional form above), each pair within rc once, minimum image.  The list (radius rc +
 * skin, the cells of a SW list of radius rcs, a +-2 cell stencil) is built inside the call.
 *   x, n, box   device FP64 SoA [3n] positions, atoms, host box [3]; every box length must be
 *               >= 2 (rc + skin) and give >= 5 cells of width >= rcs.
 *   rcs, skin   cell criterion and list skin (rc + skin <= 2 rcs).
 *   uf          host, UF parameters.
 *   precision   NEFE_FP32 or NEFE_FP64 pair arithmetic (sums in fixed point, order independent).
 *   f           device out FP64 SoA [3n]; e_atom device out [n] or NULL (half of each pair);
 *   energy_virial device out [7] or NULL: E and the virial xx yy zz xy xz yz.
 * Scratch is allocated stream-ordered and released on the stream.  Returns NEFE_EINVAL on bad
 * arguments, NEFE_EOVERFLOW when a row exceeds NEFE_UF_CAP, NEFE_ENOMEM / NEFE_ECUDA.
 * Blocking: yes (reads the overflow flag).
 */
NEFE_API int nefe_uf_forces(const double* x, int n, const double box[3], double rcs, double skin,
                            const nefe_uf_params* uf, int precision, double* f, double* e_atom,
                            double* energy_virial, void* stream);

/*
 * nefe_sw_energy_grad - the SW energy, forces and the derivatives of the energy with respect to
 * the potential parameters theta = (A, B, p, q, a, lambda3, gamma) (eps, sigma, cos0 fixed), for
 * differentiating the model (the backward of an energy function).  Pair terms give
 *   dE/dA = E2/A, dE/dB = eps A s^-p e, dE/dp = -eps A B s^-p ln(s) e, dE/dq = eps A s^-q ln(s) e,
 *   dE/da = sum phi2/(s-a)^2 + sum h gamma (1/(s_ij-a)^2 + 1/(s_ik-a)^2)
 * with e = exp(1/(s-a)); triplet terms dE/dlambda3 = sum h/lambda3, dE/dgamma =
 * sum h (1/(s_ij-a) + 1/(s_ik-a)).  Same list and layout rules as nefe_sw_forces.
 *   f            device out FP64 SoA [3n] forces, or NULL.
 *   energy_grad  device out FP64 [8]: E, then dE/dA, dE/dB, dE/dp, dE/dq, dE/da, dE/dlambda3,
 *                dE/dgamma (each summed in fixed point, decoded in FP64).
 * Returns NEFE_EOVERFLOW when an atom has more than 32 neighbours inside a*sigma, NEFE_ENAN on
 * a non-finite sum, NEFE_EINVAL on bad arguments, NEFE_ENOMEM / NEFE_ECUDA.  Blocking: yes (it reads the
 * error word back).
 */
NEFE_API int nefe_sw_energy_grad(const double* x, int n, const double box[3], double rcs,
                                 const int* nbr, const int* cnt, int cap, const nefe_sw_params* prm,
                                 int precision, double* f, double* energy_grad, void* stream);

/*
 * nefe_langevin_noise - the standard-normal thermostat noise the integrator draws for
 * atoms 0..n-1 of system `sys_id` at step `step`: Philox4x64-10 (Salmon et al., SC'11) with
 * counter (step, atom, sys_id, 0) and key (seed, 0), two Box-Muller pairs from the four
 * outputs, first three normals as x, y, z.  precision selects the FP32 or FP64 transform
 * (the integer stream is identical).  xi: device out, FP64 (n, 3) row-major.
 */
NEFE_API int nefe_langevin_noise(uint64_t seed, uint64_t sys_id, uint64_t step, int n, int precision,
                        double* xi, void* stream);

/* ---------------------------------------------------------------- engine (context API) */
typedef struct nefe_ctx nefe_ctx;

#define NEFE_POT_SW       0   /* U_int = Stillinger-Weber                                */
#define NEFE_POT_EINSTEIN 1   /* U_int = k_int/2 sum |x - r0|^2 (closed-form test system; */
                              /*   k_int = 0 is the ideal gas)                             */
#define NEFE_POT_UF       2   /* U_int = Uhlenbeck-Ford fluid (nefe_set_uf_params)         */


#define NEFE_BARO_NONE  0
#define NEFE_BARO_ISO   1
#define NEFE_BARO_ANISO 2

#define NEFE_SCHED_NONE 0     /* lambda fixed                                             */
#define NEFE_SCHED_FL   1     /* H = K + (1-l) U_int + l U_E, l = t^5(70t^4-315t^3+540t^2 */
                              /*   -420t+126), U_E = k_E/2 sum |x - r0|^2 (Sec. 2.1)      */
#define NEFE_SCHED_RS   2     /* H = K + l U_int + l P V, l = 1/(1 + t (1/l_f - 1))        */
                              /*   (Sec. 2.2 and the Sec. 4 lambda variable)               */
#define NEFE_SCHED_AS   3     /* barostat P driven P0 -> P1 linearly, dH/dP = V (Sec. 2.3) */

#define NEFE_DCCI_TEMP  0     /* temperature control: Eq. Ps_coex_discreted               */
#define NEFE_DCCI_PRESS 1     /* pressure control: Eq. l_coex_discreted                   */

/* A system (one periodic cell).  All host arrays are copied; the caller keeps ownership. */
typedef struct nefe_system_desc {
    int n;                     /* atoms, >= 2                                             */
    const double* x;           /* host (n,3) positions (A), unwrapped                     */
    const double* v;           /* host (n,3) velocities (A/ps) or NULL for zero            */
    const double* r0;          /* host (n,3) Einstein lattice sites or NULL (= x)          */
    double box[3];             /* orthorhombic box lengths (A)                             */
    double mass;               /* g/mol (all atoms)                                        */
    int pot;                   /* NEFE_POT_*                                               */
    double k_int;              /* spring of U_int when pot == NEFE_POT_EINSTEIN (eV/A^2)   */
} nefe_system_desc;

/* Switching schedule of one system (tau = min(k / nsteps, 1); direction -1 uses 1 - tau). */
typedef struct nefe_schedule {
    int kind;                  /* NEFE_SCHED_*                                             */
    int direction;             /* +1 forward, -1 backward                                  */
    long nsteps;               /* switching length in steps                                */
    double k_E;                /* FL: Einstein spring (eV/A^2)                              */
    double lambda_f;           /* RS: final lambda of the forward path                     */
    double P_GPa;              /* RS: physical pressure P (target is lambda P)              */
    double P0_GPa, P1_GPa;     /* AS: pressure path                                        */
    double lambda0;            /* NONE: fixed lambda (force scale on U_int)                 */
    int ref;                   /* FL: NEFE_REF_EINSTEIN (springs k_E about r0) or NEFE_REF_UF */
                               /*   (the system's UF parameters); 0 = Einstein              */
} nefe_schedule;

/* Results of one system after the last completed step (FP64).  H and dH/dl follow the
 * system's schedule (FL: U_E - U_int; RS: U_int + P V; AS: V; NONE: 0). */
typedef struct nefe_results {
    double W;                  /* accumulated dynamical work (eV), left-point rule         */
    double lambda;             /* current lambda (AS: current target pressure in GPa)      */
    long step;                 /* steps completed                                           */
    double U;                  /* U_int (eV), unscaled                                      */
    double U_E;                /* Einstein reference energy (eV), FL only                   */
    double K;                  /* kinetic energy (eV)                                       */
    double T;                  /* 2K / ((3N-3) kB) (K)                                      */
    double P[6];               /* pressure tensor xx,yy,zz,xy,xz,yz (GPa)                   */
    double V;                  /* volume (A^3)                                              */
    double box[3];
    double dHdl;               /* driving force at the current step                         */
    double H;                  /* Hamiltonian value at the current step                     */
    double mean_H, mean_dHdl, mean_P, mean_V;   /* running means over completed steps       */
    double P_target;           /* barostat target (GPa): lambda P (RS), P_S (dCCI), P (AS)   */
    unsigned error;            /* NEFE_ERR_* bits                                           */
} nefe_results;

/*
 * nefe_create - new context on CUDA device `device`, issuing work on `stream` (cudaStream_t
 * as void*, NULL = a stream the context creates).  A context holds every simulated cell of a
 * study (replicas, both phases of each dCCI pair; Sec. 4 runs 10 realisations per estimate and
 * two coupled partitions for dCCI) and advances them together.  precision: NEFE_FP32 /
 * NEFE_FP64.  dt_ps: time step (Sec. 4 uses 1 fs = 0.001 ps).  skin: list skin (A).
 * nbr_cap: neighbour row capacity (16..64).  NEFE_EINVAL on bad arguments, NEFE_ECUDA when no
 * device is usable.  The context owns all its device memory (released by nefe_destroy).
 */
NEFE_API int nefe_create(nefe_ctx** out, int device, void* stream, int precision, double dt_ps,
                double skin, int nbr_cap);
NEFE_API int nefe_destroy(nefe_ctx* ctx);
/* Message of the most recent failure on the calling thread, whatever context or call it came
 * from (the library keeps one message per thread, not per context). */
NEFE_API const char* nefe_last_error(void);

/* Adds a system (one periodic cell of Sec. 4: Si-cd, beta-Sn or liquid) before the first
 * nefe_run; *sys_id receives its index (0, 1, ...).  The host arrays of desc are copied.
 * NEFE_EINVAL on n < 2, NULL x or a non-positive box; NEFE_ESTATE after setup. */
NEFE_API int nefe_add_system(nefe_ctx* ctx, const nefe_system_desc* desc, int* sys_id);
/* Potential parameters for one system, or all systems when sys == -1. */
NEFE_API int nefe_set_sw_params(nefe_ctx* ctx, int sys, const nefe_sw_params* prm);
/* Uhlenbeck-Ford parameters of one system (used when its pot is NEFE_POT_UF or its FL
 * reference is NEFE_REF_UF).  Default: p = 25, sigma = 2.0 A, T = 2200 K, rc = 8.0 A.
 * NEFE_EINVAL on p <= 0, sigma <= 0, T <= 0 or rc <= 0; NEFE_ESTATE after setup.  The
 * cutoff condition rc + skin <= 2 (a sigma + skin) is checked by nefe_setup. */
NEFE_API int nefe_set_uf_params(nefe_ctx* ctx, int sys, const nefe_uf_params* uf);
/* Langevin thermostat: T (K), damping time (ps; <= 0 switches it off), noise seed.
 * The random force of each step has its per-system mean removed ("zero yes", Sec. 4). */
NEFE_API int nefe_set_thermostat(nefe_ctx* ctx, int sys, double T, double damp_ps, uint64_t seed);
/* Box equation (Sec. 4: "Parrinello-Rahman", LAMMPS fix nph iso for Si-cd and the liquid, aniso for
 * beta-Sn, with the "ners" tag that multiplies the target by lambda in reversible scaling):
 * mode NEFE_BARO_*, target pressure (GPa; the physical P of an RS schedule is set there
 * instead), damping time tau_P (ps): box mass Q_b = (N + 1) kB T tau_P^2.  The box equation is
 * a reading (the paper prints none): eta' = d V (P - P_target) / Q_b with d = 3 (iso, one
 * strain rate) or d = 1 per axis driven by P_aa (aniso), affine drift of the positions.
 * NEFE_EINVAL on a bad mode or pdamp <= 0; NEFE_ESTATE after setup. */
NEFE_API int nefe_set_barostat(nefe_ctx* ctx, int sys, int mode, double P_GPa, double pdamp_ps);
/* Switching path of one system (NEFE_SCHED_*): Hamiltonian interpolation to the Einstein crystal
 * (Sec. 2.1, Eqs. H_lambda, Wrev_HI), reversible scaling (Sec. 2.2, Eqs. H_RS, dH_RS, with the
 * Sec. 4 lambda variable), pressure switching (Sec. 2.3, Eqs. Wmech, Wmech_dyn), or a fixed
 * lambda.  The work W = sum_k dH/dlambda (lambda_{k+1} - lambda_k) (Eq. Wdyn, left point) is
 * accumulated in FP64 on the device.  NEFE_EINVAL on an unknown kind or nsteps < 1;
 * NEFE_ESTATE after setup. */
NEFE_API int nefe_set_schedule(nefe_ctx* ctx, int sys, const nefe_schedule* sched);
/*
 * nefe_pair_dcci - couples systems sysI and sysII (phase I, phase II) through the dCCI
 * update (Sec. 3): both run at fixed T0 with barostats (set separately) whose common
 * target P_S starts at P0_GPa, and a common lambda starting at 1.  mode TEMP: T(t) runs
 * linearly from -> to (K) over nsteps, lambda = from / T(t) (T0 must equal from), P_S by Eq.
 * Ps_coex_discreted.  mode PRESS: P(t) runs from -> to (GPa), lambda by Eq.
 * l_coex_discreted, P_S = lambda P.  dU, dV are per-atom differences of phase I minus
 * phase II.  *pair_id receives the pair index.
 */
NEFE_API int nefe_pair_dcci(nefe_ctx* ctx, int sysI, int sysII, double T0, double P0_GPa, int mode,
                   double from, double to, long nsteps, int* pair_id);
/* Decimated per-system trace: every `every` steps one record of 9 doubles (step, lambda,
 * W, dH/dl, U, V, P (GPa), P_target (GPa), T) into a device ring of `cap` records. */
NEFE_API int nefe_set_trace(nefe_ctx* ctx, int sys, int every, long cap);

/* Uploads all state, builds lists and computes the initial forces (implicit in the first
 * nefe_run).  After setup, systems can no longer be added. */
NEFE_API int nefe_setup(nefe_ctx* ctx);
/* Advances every system by nsteps (asynchronous; replays a captured CUDA graph of the
 * step sequence in chunks). */
NEFE_API int nefe_run(nefe_ctx* ctx, long nsteps);
/* Blocks until the context's stream is idle; returns NEFE_ECUDA on an asynchronous error, and
 * NEFE_ETIMEOUT if a grid barrier of the list rebuild gave up waiting since the last call (its
 * systems then carry NEFE_ERR_TIMEOUT; the barrier is reset, the lists of that step are not
 * valid: reload a checkpoint or set the state again). */
NEFE_API int nefe_sync(nefe_ctx* ctx);

/* Blocking reads (they synchronise the stream first).  nefe_get_results: the dynamical work W
 * of Eq. Wdyn (left point; forward and backward runs give Eqs. dF and Qdiss on the host),
 * the instantaneous and mean H, dH/dlambda, P and V of the system (Sec. 2), lambda and the
 * error word; NEFE_EINVAL for an unknown system.  nefe_get_pair: T_coex = T0 / lambda and
 * P_coex = P_S / lambda of a dCCI pair (Sec. 3, Eqs. T_sc, P_sc). */
NEFE_API int nefe_get_results(nefe_ctx* ctx, int sys, nefe_results* out);
NEFE_API int nefe_get_pair(nefe_ctx* ctx, int pair, double* T_coex, double* P_coex_GPa,
                  double* lambda, unsigned* error);
/* Host (n,3) positions / velocities and box[3]; any pointer may be NULL. */
NEFE_API int nefe_get_state(nefe_ctx* ctx, int sys, double* x, double* v, double* box);
/* Replaces positions and velocities (host (n,3), NULL keeps) of one system; forces and
 * lists are recomputed before the next step. */
NEFE_API int nefe_set_state(nefe_ctx* ctx, int sys, const double* x, const double* v);
/* Copies up to cap records (9 doubles each, oldest first) into host buf; *n = count. */
NEFE_API int nefe_get_trace(nefe_ctx* ctx, int sys, double* buf, long cap, long* n);

/* Checkpoint: full dynamic state (positions, velocities, forces, box, barostat, lambda,
 * work, accumulators, step counters, pair state); RNG needs no state (counter-based), so a
 * resumed run is bitwise identical to an uninterrupted one. */
NEFE_API int nefe_save(nefe_ctx* ctx, const char* path);
NEFE_API int nefe_load(nefe_ctx* ctx, const char* path);

/* Times the variants of both force passes on the current state and keeps the fastest:
 * pass A with 1 (one thread per atom), 4, 8, 16 or 32 lanes per atom (FP64: 8, 16, 32),
 * pass B with 1, 2, 4 or 8 lanes per atom, and the rebuild policy (nefe_set_rebuild_policy); the
 * list build keeps its form (nefe_set_list_tuning).  Each force pass is first timed alone; then
 * the two fastest pass-A variants with every pass-B variant, and with the best pair each rebuild
 * policy, run as real steps on a device snapshot of the state, restored afterwards (the run
 * continues bit for bit as without the call; the snapshot needs about as much free device
 * memory as the state, and without it the kernel-level choice stands).  nefe_get_tuning
 * reports pass A's lanes and the time per MD step of the chosen pair (kernel-level: the two
 * passes' summed time); nefe_set_tuning fixes pass A's lanes.  Blocking. */
NEFE_API int nefe_autotune(nefe_ctx* ctx);
NEFE_API int nefe_get_tuning(nefe_ctx* ctx, int* lanes_per_atom, double* best_us);
NEFE_API int nefe_set_tuning(nefe_ctx* ctx, int lanes_per_atom);
/* Lanes per atom in use: [0] pass A, [1] pass B, [2] list build. */
NEFE_API int nefe_get_lanes(nefe_ctx* ctx, int lanes[3]);
/* Fixes pass B's lanes per atom (1, 2, 4 or 8). */
NEFE_API int nefe_set_gather_tuning(nefe_ctx* ctx, int lanes_per_atom);
/* Fixes the list build's form: 0 = one warp per cell (the default), or 8, 16, 32 lanes per atom. */
NEFE_API int nefe_set_list_tuning(nefe_ctx* ctx, int lanes_per_atom);
/* The engine's list rebuild as one cooperative launch (on = 1: worklist, cell count, scan, fill
 * and list build in one kernel whose phases are separated by time-bounded grid barriers; its
 * blocks return at once on a step without a stale list) or as the kernel sequence (on = 0, the
 * default).  Both build the same lists bit for bit.  On this GPU the cooperative node of the step
 * graph costs more per step (measured 244 against 237 us per MD step on the benchmark workload)
 * than the four launches it replaces, hence the default.  Applies when the list build runs one
 * warp per cell and no system has a Uhlenbeck-Ford term.  NEFE_EINVAL for other values. */
NEFE_API int nefe_set_cooperative_rebuild(nefe_ctx* ctx, int on);

/* Failure detection of the time-bounded grid barrier (the one device-side wait of the library,
 * in the engine's single-launch list rebuild; the paper has no counterpart).  Launches a small
 * grid whose barrier can never complete (it expects one block more than it has), with a limit of
 * limit_ms milliseconds: every block must give up, record the timeout and return, so the call
 * returns NEFE_ETIMEOUT and the device stays usable.  NEFE_OK would mean the wait did not end by
 * its limit (never expected); NEFE_EINVAL for limit_ms outside (0, 1000]. */
NEFE_API int nefe_check_barrier_timeout(int device, double limit_ms);

/* Rebuild policy of the Verlet lists (the skin criterion of the list, Sec. 4's MD setup; the
 * paper itself does not discuss lists).  all = 0: each system rebuilds when one of its own atoms
 * has moved more than skin/2 since its last build.  all = 1: on a step where any system needs
 * a rebuild, every system rebuilds -- lists are rebuilt earlier than needed, which never
 * changes what the force passes compute (trajectories differ from policy 0 only by the
 * rounding of the position anchor), and the batch then runs one full-width build instead of
 * many narrow ones.  nefe_autotune times both in real steps and keeps the faster.
 * NEFE_EINVAL for other values.  nefe_get_rebuild_policy: the policy in use. */
NEFE_API int nefe_set_rebuild_policy(nefe_ctx* ctx, int all);
NEFE_API int nefe_get_rebuild_policy(nefe_ctx* ctx, int* all);

/* Batched state transfer for every system at once: host (Ntot, 3) arrays, systems in the
 * order they were added (Ntot = sum of their n).  One host<->device copy each, the layout
 * change runs on the device.  set_state_all recomputes lists and forces like
 * nefe_set_state.  Any pointer may be NULL (kept / not read). */
NEFE_API int nefe_set_state_all(nefe_ctx* ctx, const double* x, const double* v);
NEFE_API int nefe_get_state_all(nefe_ctx* ctx, double* x, double* v);
/* Results of the first `count` systems into out[0..count). */
NEFE_API int nefe_get_results_all(nefe_ctx* ctx, nefe_results* out, int count);

/* Neighbour-list statistics of one system (sys >= 0) or of all (sys == -1): mean and maximum
 * row length and the number of list builds so far (the initial build included). */
NEFE_API int nefe_get_list_stats(nefe_ctx* ctx, int sys, double* mean_count, int* max_count,
                                 long* builds);

/* In-cutoff shell statistics of the SW systems after the last force evaluation: mean and maximum
 * number of neighbours inside the active cutoff per atom.  Blocking. */
NEFE_API int nefe_get_shell_stats(nefe_ctx* ctx, double* mean_count, int* max_count);

/* Kernel timing: with profiling enabled, the captured step graph records CUDA events around
 * the two force passes of every step; nefe_get_profile writes the mean time per step (us)
 * of pass A (edges: pair terms and triplets) to us[0] and of pass B (gather, springs,
 * Langevin, half kick) to us[1] over the steps of the most recent graph replay (each summed
 * over the L2-sized chunks the passes run in), and the number of steps averaged.
 * Blocking. */
NEFE_API int nefe_set_profiling(nefe_ctx* ctx, int enable);
NEFE_API int nefe_get_profile(nefe_ctx* ctx, double* us, long* samples);

/* Number of kernel launches the context issued so far (for launch accounting). */
NEFE_API int nefe_launch_count(nefe_ctx* ctx, long* count);

/* ------------------------------------------------------------------------------------------
 * Differentiation of the switching work (the W adjoint).
 *
 * W(theta) = sum_k dH/dlambda(x_k) (lambda_{k+1} - lambda_k) (Eq. Wdyn, left point) along an
 * FP64 NVT Langevin velocity-Verlet trajectory (Frenkel-Ladd: dH/dlambda = U_E - U_SW, Sec. 2.1;
 * reversible scaling: dH/dlambda = U_SW + P V, Sec. 2.2), as a function of the SW parameters
 * theta = (A, B, p, q, a, lambda3, gamma) and of the initial state, with the thermostat noise
 * (same Philox stream as the engine) held fixed.  The update is the engine's: half kick, drift,
 * F = s_int F_SW + s_E F_E - (m/tdamp) v_half + amp (xi - mean xi), half kick.
 * ------------------------------------------------------------------------------------------ */

/*
 * nefe_sw_dual - SW energy, forces and dU/dtheta in FP64 dual numbers: the dual direction is
 * the displacement w of every atom together with the parameter direction dtheta.  Gives the
 * Hessian-vector product J w (J = dF/dx) and the mixed product (d2U/dtheta dx) w.
 *   x, w      device in FP64 SoA [3n] (w may be NULL: zero)
 *   nbr, cnt  a list from nefe_neighbor_build with rcs >= a*sigma (minimum image is taken on
 *             the box, so box >= 2 rcs as there)
 *   dtheta    host [7] parameter direction, or NULL (zero)
 *   f, fd     device out FP64 SoA [3n]: F and its dual part J w + (dF/dtheta) dtheta
 *   out16     device out FP64 [16]: E, E' = -F.w + G.dtheta, G = dU/dtheta [7], G' [7]
 * Returns NEFE_EOVERFLOW (shell above 32), NEFE_ENAN, NEFE_EINVAL, NEFE_ECUDA.  Blocking: yes.
 */
NEFE_API int nefe_sw_dual(const double* x, const double* w, int n, const double box[3], double rcs,
                          const int* nbr, const int* cnt, int cap, const nefe_sw_params* prm,
                          const double* dtheta, double* f, double* fd, double* out16, void* stream);

typedef struct nefe_adj nefe_adj;

typedef struct nefe_adjoint_desc {
    int n;                     /* atoms                                                     */
    const double* x;           /* host (n, 3) initial positions, A (copied at create)       */
    const double* v;           /* host (n, 3) initial velocities, A/ps                      */
    const double* r0;          /* host (n, 3) Einstein sites (FL), or NULL (RS)             */
    double box[3];             /* orthorhombic periodic box, A (fixed: NVT), >= 2 rcs       */
    double mass;               /* g/mol                                                     */
    double dt;                 /* ps                                                        */
    double T;                  /* K                                                         */
    double tdamp;              /* ps; <= 0: no thermostat                                   */
    uint64_t seed, sys_id;     /* noise stream                                              */
    int kind;                  /* NEFE_SCHED_FL or NEFE_SCHED_RS                            */
    int direction;             /* +1 forward, -1 backward                                   */
    long nsched;               /* switching steps: tau = min(k / nsched, 1)                 */
    double k_E;                /* FL spring, eV/A^2                                         */
    double lambda_f;           /* RS end point                                              */
    double P_GPa;              /* RS: external pressure in the P V term                     */
    double skin;               /* list radius rcs = a sigma + skin, A                       */
    int nbr_cap;               /* neighbour row capacity, 1..64                             */
    int checkpoint_every;      /* K_c: (x, v, F) kept every K_c steps, >= 1                 */
} nefe_adjoint_desc;

/* Creates the context on `device` / `stream` (device memory ~ (17 + 3 K_c) n doubles plus
 * 9 n doubles per checkpoint).  NEFE_EINVAL on bad arguments, NEFE_ENOMEM. */
NEFE_API int nefe_adjoint_create(nefe_adj** out, int device, void* stream, const nefe_adjoint_desc* desc,
                                 const nefe_sw_params* prm);
NEFE_API int nefe_adjoint_destroy(nefe_adj* adj);
/* Replaces the SW parameters (a*sigma must stay within the list radius fixed at create);
 * invalidates the checkpoints. */
NEFE_API int nefe_adjoint_set_params(nefe_adj* adj, const nefe_sw_params* prm);
/* Runs nsteps from the initial state, keeping the checkpoints; *W (host) = the work.  The neighbour
 * list is rebuilt at every force evaluation.  Blocking.  NEFE_EOVERFLOW / NEFE_ENAN on a bad run. */
NEFE_API int nefe_adjoint_forward(nefe_adj* adj, long nsteps, double* W);
/* Reverse sweep over the last forward run: dW/dtheta (host [7]) and, when not NULL, dW/dx0 and
 * dW/dv0 (host (n, 3)).  Each segment is recomputed from its checkpoint.  Blocking.
 * NEFE_ESTATE without a preceding forward run. */
NEFE_API int nefe_adjoint_backward(nefe_adj* adj, double dW_dtheta[7], double* dW_dx0, double* dW_dv0);
/* Tangent-linear run: W and its directional derivative dW along (dtheta [7], dx0, dv0 (n, 3) host
 * or NULL).  Invalidates the checkpoints.  Blocking. */
NEFE_API int nefe_adjoint_tangent(nefe_adj* adj, long nsteps, const double dtheta[7], const double* dx0,
                                  const double* dv0, double* W, double* dW);
/* Positions and velocities (host (n, 3), either may be NULL) at the end of the last run. */
NEFE_API int nefe_adjoint_state(nefe_adj* adj, double* x, double* v);

#ifdef __cplusplus
}
#endif
#endif /* NEFE_H */
