/*
 * FP64 CPU oracle for the Stillinger-Weber / non-equilibrium free-energy hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct definition that the
 * CUDA library is checked against.  Only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark may load it.  It shares no code, header, table or constant generator
 * with the CUDA library under paper_2103_10449_gb300/csrc, and it never includes anything
 * from there.
 *
 * Contents (each routine states what it follows):
 *   orc_philox4x64      Philox4x64-10 counter-based generator (Salmon, Moraes, Dror, Shaw,
 *                       "Parallel random numbers: as easy as 1, 2, 3", SC'11), written from
 *                       the published round function and constants.
 *   orc_langevin_xi     Gaussian thermostat noise drawn from that generator (Box-Muller).
 *   orc_sw_energy       Stillinger-Weber energy, forces and virial by brute force over all
 *                       atom pairs with the minimum-image convention (the potential the paper
 *                       uses for Si, Sec. 4; functional form of Stillinger & Weber 1985).
 *   orc_sw_force_atoms  The same forces for a chosen subset of atoms (sampled parity at sizes
 *                       where the all-atom O(N^2) loop is too slow).
 *   orc_neighbor_list   Verlet list by brute force: every j != i whose minimum-image
 *                       distance squared is strictly below (rc + skin)^2, rows ordered by j.
 *   orc_cell_bin        Cell assignment and the stable counting sort by (cell, atom index).
 *   orc_uf_energy       Uhlenbeck-Ford pair energy, forces and virial by brute force (the
 *                       fluid reference system the paper uses for the liquid, Sec. 2.1 and
 *                       Sec. 4, from Paula Leite et al. 2016), truncated and shifted at rc.
 *
 * All floating-point arithmetic is IEEE binary64; build with -ffp-contract=off so that no
 * multiply-add is fused (the integer decisions of the list and the cells then follow the
 * plain left-to-right evaluation written here).
 *
 * Parameter vector layout used by orc_sw_* (10 doubles):
 *   [0] epsilon (eV)  [1] sigma (A)  [2] A  [3] B  [4] p  [5] q  [6] a (cutoff in sigma)
 *   [7] lambda3       [8] gamma      [9] cos(theta0)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------------------ */
/* Philox4x64-10 (SC'11).  Round: (hi0,lo0) = M0*X0, (hi1,lo1) = M1*X2,                  */
/* X <- (hi1 ^ X1 ^ k0, lo1, hi0 ^ X3 ^ k1, lo0); key bumped by the Weyl constants.     */
/* ------------------------------------------------------------------------------------ */
static void mulhilo64(uint64_t a, uint64_t b, uint64_t* hi, uint64_t* lo) {
    unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
    *hi = (uint64_t)(p >> 64);
    *lo = (uint64_t)p;
}

void orc_philox4x64(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
    uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t hi0, lo0, hi1, lo1;
        mulhilo64(M0, x0, &hi0, &lo0);
        mulhilo64(M1, x2, &hi1, &lo1);
        uint64_t n0 = hi1 ^ x1 ^ k0, n1 = lo1, n2 = hi0 ^ x3 ^ k1, n3 = lo0;
        x0 = n0; x1 = n1; x2 = n2; x3 = n3;
        k0 += W0; k1 += W1;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Open-interval uniform (0,1) from the top 53 bits. */
static double u01(uint64_t r) { return ((double)(r >> 11) + 0.5) * (1.0 / 9007199254740992.0); }

/*
 * Thermostat noise: for atom `id` of system `sys` at integration step `step` the counter is
 * (step, id, sys, 0) and the key (seed, 0).  Two Box-Muller pairs are formed from the four
 * 64-bit outputs; the first three normals are the x, y, z components.
 */
void orc_langevin_xi(uint64_t seed, uint64_t sys, uint64_t step, int64_t n, double* xi) {
    const double two_pi = 6.283185307179586476925286766559;
    for (int64_t i = 0; i < n; ++i) {
        uint64_t ctr[4] = {step, (uint64_t)i, sys, 0};
        uint64_t key[2] = {seed, 0};
        uint64_t r[4];
        orc_philox4x64(ctr, key, r);
        double rho0 = sqrt(-2.0 * log(u01(r[0])));
        double th0 = two_pi * u01(r[1]);
        double rho1 = sqrt(-2.0 * log(u01(r[2])));
        double th1 = two_pi * u01(r[3]);
        xi[3 * i + 0] = rho0 * cos(th0);
        xi[3 * i + 1] = rho0 * sin(th0);
        xi[3 * i + 2] = rho1 * cos(th1);
    }
}

/* ------------------------------------------------------------------------------------ */
/* Minimum image: raw = xj - xi; m = rint(raw / L); d = raw - m * L.                     */
/* ------------------------------------------------------------------------------------ */
static double min_image(double xj, double xi, double L, double* m_out) {
    double raw = xj - xi;
    double m = rint(raw / L);
    double mL = m * L;
    if (m_out) *m_out = m;
    return raw - mL;
}

/* Stillinger-Weber pieces in reduced distance s = r / sigma (Stillinger & Weber 1985):   */
/*   f2(s) = A (B s^-p - s^-q) exp(1/(s - a))       for s < a                            */
/*   h(s_ij, s_ik, c) = lambda3 (c - c0)^2 exp(gamma/(s_ij - a)) exp(gamma/(s_ik - a))   */
/* Energies carry the factor epsilon.                                                    */
typedef struct { double eps, sig, A, B, p, q, a, lam, gam, c0; } swp;
static swp unpack(const double* prm) {
    swp s = {prm[0], prm[1], prm[2], prm[3], prm[4], prm[5], prm[6], prm[7], prm[8], prm[9]};
    return s;
}

/* phi2(r) and dphi2/dr, r in Angstrom. */
static void pair_term(const swp* P, double r, double* phi, double* dphi) {
    double s = r / P->sig;
    double rp = pow(s, -P->p), rq = pow(s, -P->q);
    double ex = exp(1.0 / (s - P->a));
    double poly = P->B * rp - rq;
    double dpoly = (-P->p * P->B * rp + P->q * rq) / s;
    double dex = -ex / ((s - P->a) * (s - P->a));
    *phi = P->eps * P->A * poly * ex;
    *dphi = P->eps * P->A * (dpoly * ex + poly * dex) / P->sig;
}

/* g(r) = exp(gamma/(s - a)) and dg/dr. */
static void leg_term(const swp* P, double r, double* g, double* dg) {
    double s = r / P->sig;
    double den = s - P->a;
    *g = exp(P->gam / den);
    *dg = -(*g) * P->gam / (den * den) / P->sig;
}

typedef struct { int64_t j; double d[3]; double r; } nb_t;

/* Per-atom list of neighbours inside the potential cutoff a*sigma (brute force). */
static int build_cut_lists(int64_t n, const double* x, const double* box, double rc,
                           int cap, nb_t* nb, int* cnt) {
    for (int64_t i = 0; i < n; ++i) {
        int c = 0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double d0 = min_image(x[3 * j + 0], x[3 * i + 0], box[0], NULL);
            double d1 = min_image(x[3 * j + 1], x[3 * i + 1], box[1], NULL);
            double d2 = min_image(x[3 * j + 2], x[3 * i + 2], box[2], NULL);
            double rr = d0 * d0 + d1 * d1 + d2 * d2;
            if (rr < rc * rc) {
                if (c >= cap) return -1;
                nb_t* e = &nb[i * cap + c];
                e->j = j; e->d[0] = d0; e->d[1] = d1; e->d[2] = d2; e->r = sqrt(rr);
                ++c;
            }
        }
        cnt[i] = c;
    }
    return 0;
}

/*
 * Energy of the whole system:
 *   E = sum_{i<j} eps f2(r_ij/sigma) + sum_i sum_{j<k} eps h(r_ij, r_ik, cos theta_jik)
 * with j, k ranging over the neighbours of i inside a*sigma.  Forces are the analytic
 * -dE/dx.  Virial tensor W_ab = sum over every term of sum_legs (x_leg - x_centre)_a f_leg_b,
 * which for a pair is r_ij (x) f_j.  Per-atom energies give half of each pair term to each
 * partner and each three-body term to its centre atom.  Box lengths must exceed 2 a sigma.
 * Returns E, or NaN when the box is too small or a neighbour shell overflows.
 */
double orc_sw_energy(int64_t n, const double* x, const double* box, const double* prm,
                     double* f, double* vir, double* eatom) {
    swp P = unpack(prm);
    double rc = P.a * P.sig;
    for (int k = 0; k < 3; ++k) if (!(box[k] > 2.0 * rc)) return NAN;
    const int cap = 128;
    nb_t* nb = (nb_t*)malloc(sizeof(nb_t) * (size_t)cap * (size_t)(n > 0 ? n : 1));
    int* cnt = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    if (build_cut_lists(n, x, box, rc, cap, nb, cnt) != 0) { free(nb); free(cnt); return NAN; }
    double E = 0.0, W[9] = {0};
    if (f) memset(f, 0, sizeof(double) * 3 * (size_t)n);
    if (eatom) memset(eatom, 0, sizeof(double) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        /* two-body: each unordered pair once (j > i) */
        for (int a = 0; a < cnt[i]; ++a) {
            const nb_t* e = &nb[i * cap + a];
            if (e->j <= i) continue;
            double phi, dphi;
            pair_term(&P, e->r, &phi, &dphi);
            E += phi;
            if (eatom) { eatom[i] += 0.5 * phi; eatom[e->j] += 0.5 * phi; }
            double fj[3];
            for (int k = 0; k < 3; ++k) fj[k] = -dphi * e->d[k] / e->r; /* force on j */
            if (f) for (int k = 0; k < 3; ++k) { f[3 * e->j + k] += fj[k]; f[3 * i + k] -= fj[k]; }
            for (int p = 0; p < 3; ++p) for (int q = 0; q < 3; ++q) W[3 * p + q] += e->d[p] * fj[q];
        }
        /* three-body centred at i: unordered neighbour pairs (j, k) */
        for (int a = 0; a < cnt[i]; ++a) {
            for (int b = a + 1; b < cnt[i]; ++b) {
                const nb_t* ej = &nb[i * cap + a];
                const nb_t* ek = &nb[i * cap + b];
                double rj = ej->r, rk = ek->r;
                double uj[3], uk[3];
                for (int k = 0; k < 3; ++k) { uj[k] = ej->d[k] / rj; uk[k] = ek->d[k] / rk; }
                double c = uj[0] * uk[0] + uj[1] * uk[1] + uj[2] * uk[2];
                double gj, dgj, gk, dgk;
                leg_term(&P, rj, &gj, &dgj);
                leg_term(&P, rk, &gk, &dgk);
                double dc = c - P.c0;
                double h = P.eps * P.lam * dc * dc * gj * gk;
                E += h;
                if (eatom) eatom[i] += h;
                /* dh/dx_j = eps lam [2 dc gj gk (uk - c uj)/rj + dc^2 dgj gk uj] */
                double fj[3], fk[3];
                for (int k = 0; k < 3; ++k) {
                    double dhj = P.eps * P.lam * (2.0 * dc * gj * gk * (uk[k] - c * uj[k]) / rj
                                                  + dc * dc * dgj * gk * uj[k]);
                    double dhk = P.eps * P.lam * (2.0 * dc * gj * gk * (uj[k] - c * uk[k]) / rk
                                                  + dc * dc * gj * dgk * uk[k]);
                    fj[k] = -dhj;
                    fk[k] = -dhk;
                }
                if (f) for (int k = 0; k < 3; ++k) {
                    f[3 * ej->j + k] += fj[k];
                    f[3 * ek->j + k] += fk[k];
                    f[3 * i + k] -= fj[k] + fk[k];
                }
                for (int p = 0; p < 3; ++p) for (int q = 0; q < 3; ++q)
                    W[3 * p + q] += ej->d[p] * fj[q] + ek->d[p] * fk[q];
            }
        }
    }
    if (vir) {  /* symmetric tensor as xx, yy, zz, xy, xz, yz */
        vir[0] = W[0]; vir[1] = W[4]; vir[2] = W[8];
        vir[3] = 0.5 * (W[1] + W[3]); vir[4] = 0.5 * (W[2] + W[6]); vir[5] = 0.5 * (W[5] + W[7]);
    }
    free(nb); free(cnt);
    return E;
}

/*
 * Forces on the atoms listed in idx[0..ns) only, from every term that involves them
 * (pair terms, three-body terms centred on them and three-body terms in which they are a
 * leg).  Neighbour shells are found by brute force over all n atoms, so the cost is
 * O(ns * n + ns * shell^2).  Returns 0, or -1 when the box is too small / a shell overflows.
 */
int orc_sw_force_atoms(int64_t n, const double* x, const double* box, const double* prm,
                       int64_t ns, const int64_t* idx, double* fout) {
    swp P = unpack(prm);
    double rc = P.a * P.sig;
    for (int k = 0; k < 3; ++k) if (!(box[k] > 2.0 * rc)) return -1;
    enum { CAP = 128 };
    nb_t shell_i[CAP], shell_j[CAP];
    for (int64_t s = 0; s < ns; ++s) {
        int64_t i = idx[s];
        int ci = 0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double d0 = min_image(x[3 * j + 0], x[3 * i + 0], box[0], NULL);
            double d1 = min_image(x[3 * j + 1], x[3 * i + 1], box[1], NULL);
            double d2 = min_image(x[3 * j + 2], x[3 * i + 2], box[2], NULL);
            double rr = d0 * d0 + d1 * d1 + d2 * d2;
            if (rr < rc * rc) {
                if (ci >= CAP) return -1;
                shell_i[ci].j = j; shell_i[ci].d[0] = d0; shell_i[ci].d[1] = d1;
                shell_i[ci].d[2] = d2; shell_i[ci].r = sqrt(rr); ++ci;
            }
        }
        double F[3] = {0, 0, 0};
        for (int a = 0; a < ci; ++a) {           /* pair terms */
            double phi, dphi;
            pair_term(&P, shell_i[a].r, &phi, &dphi);
            for (int k = 0; k < 3; ++k) F[k] += dphi * shell_i[a].d[k] / shell_i[a].r;
        }
        for (int a = 0; a < ci; ++a) {           /* three-body centred at i */
            for (int b = a + 1; b < ci; ++b) {
                double rj = shell_i[a].r, rk = shell_i[b].r, uj[3], uk[3];
                for (int k = 0; k < 3; ++k) { uj[k] = shell_i[a].d[k] / rj; uk[k] = shell_i[b].d[k] / rk; }
                double c = uj[0] * uk[0] + uj[1] * uk[1] + uj[2] * uk[2];
                double gj, dgj, gk, dgk;
                leg_term(&P, rj, &gj, &dgj);
                leg_term(&P, rk, &gk, &dgk);
                double dc = c - P.c0;
                for (int k = 0; k < 3; ++k) {
                    double dhj = P.eps * P.lam * (2.0 * dc * gj * gk * (uk[k] - c * uj[k]) / rj
                                                  + dc * dc * dgj * gk * uj[k]);
                    double dhk = P.eps * P.lam * (2.0 * dc * gj * gk * (uj[k] - c * uk[k]) / rk
                                                  + dc * dc * gj * dgk * uk[k]);
                    F[k] += dhj + dhk;          /* f_i = -(f_j + f_k) = dh/dx_j + dh/dx_k */
                }
            }
        }
        for (int a = 0; a < ci; ++a) {           /* three-body centred at neighbour j, i a leg */
            int64_t j = shell_i[a].j;
            int cj = 0;
            for (int64_t k2 = 0; k2 < n; ++k2) {
                if (k2 == j) continue;
                double d0 = min_image(x[3 * k2 + 0], x[3 * j + 0], box[0], NULL);
                double d1 = min_image(x[3 * k2 + 1], x[3 * j + 1], box[1], NULL);
                double d2 = min_image(x[3 * k2 + 2], x[3 * j + 2], box[2], NULL);
                double rr = d0 * d0 + d1 * d1 + d2 * d2;
                if (rr < rc * rc) {
                    if (cj >= CAP) return -1;
                    shell_j[cj].j = k2; shell_j[cj].d[0] = d0; shell_j[cj].d[1] = d1;
                    shell_j[cj].d[2] = d2; shell_j[cj].r = sqrt(rr); ++cj;
                }
            }
            /* leg j->i is d_ji = -d_ij */
            double rji = shell_i[a].r, uji[3];
            for (int k = 0; k < 3; ++k) uji[k] = -shell_i[a].d[k] / rji;
            double gi, dgi;
            leg_term(&P, rji, &gi, &dgi);
            for (int b = 0; b < cj; ++b) {
                if (shell_j[b].j == i) continue;
                double rk = shell_j[b].r, uk[3];
                for (int k = 0; k < 3; ++k) uk[k] = shell_j[b].d[k] / rk;
                double c = uji[0] * uk[0] + uji[1] * uk[1] + uji[2] * uk[2];
                double gk, dgk;
                leg_term(&P, rk, &gk, &dgk);
                double dc = c - P.c0;
                for (int k = 0; k < 3; ++k) {
                    double dhi = P.eps * P.lam * (2.0 * dc * gi * gk * (uk[k] - c * uji[k]) / rji
                                                  + dc * dc * dgi * gk * uji[k]);
                    F[k] -= dhi;                /* f_i = -dh/dx_i */
                }
            }
        }
        for (int k = 0; k < 3; ++k) fout[3 * s + k] = F[k];
    }
    return 0;
}

/*
 * Verlet list by brute force.  For each i, every j != i (ascending j) with
 *   d = min-image(x_j - x_i),  d.d < rcs^2   (strict)
 * is listed; img receives the integer image shift m per axis (d = x_j - x_i - m L).
 * d.d is evaluated as ((dx*dx + dy*dy) + dz*dz).  Requires every box length >= 2 rcs so
 * that at most one image of j lies within rcs.  Returns 0, -1 on overflow of cap (cnt then
 * holds the true count), -2 when the box is too small.
 */
int orc_neighbor_list(int64_t n, const double* x, const double* box, double rcs, int cap,
                      int32_t* nbr, int32_t* cnt, int32_t* img) {
    for (int k = 0; k < 3; ++k) if (!(box[k] >= 2.0 * rcs)) return -2;
    int rc = 0;
    double rcs2 = rcs * rcs;
    for (int64_t i = 0; i < n; ++i) {
        int c = 0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double m[3];
            double d0 = min_image(x[3 * j + 0], x[3 * i + 0], box[0], &m[0]);
            double d1 = min_image(x[3 * j + 1], x[3 * i + 1], box[1], &m[1]);
            double d2 = min_image(x[3 * j + 2], x[3 * i + 2], box[2], &m[2]);
            double rr = d0 * d0 + d1 * d1;
            rr = rr + d2 * d2;
            if (rr < rcs2) {
                if (c < cap) {
                    nbr[i * cap + c] = (int32_t)j;
                    if (img) for (int k = 0; k < 3; ++k) img[(i * cap + c) * 3 + k] = (int32_t)m[k];
                }
                ++c;
            }
        }
        cnt[i] = c;
        if (c > cap) rc = -1;
    }
    return rc;
}

/*
 * Cell grid and cell assignment.  Per axis, ncell = floor(L / rcs), reduced by one while
 * L / ncell < rcs * (1 + 1e-9) (cells strictly wider than rcs).  An atom's wrapped
 * fractional coordinate is w = x/L - floor(x/L), its cell index c = (int)(w * ncell),
 * clamped to ncell - 1; the linear cell id is cx + nx (cy + ny cz).  cell_start/perm are the
 * stable counting sort of the atoms by cell id (ties by atom index).  Returns the number
 * of cells, or -1 when a box length gives fewer than 2 cells or ncell_cap is too small.
 */
int orc_cell_bin(int64_t n, const double* x, const double* box, double rcs, int ncell_cap,
                 int32_t* ncell3, int32_t* cell_of, int32_t* cell_start, int32_t* perm) {
    int nc[3];
    for (int k = 0; k < 3; ++k) {
        int m = (int)floor(box[k] / rcs);
        while (m > 0 && box[k] / (double)m < rcs * (1.0 + 1e-9)) --m;
        if (m < 2) return -1;
        nc[k] = m;
        ncell3[k] = m;
    }
    long total = (long)nc[0] * nc[1] * nc[2];
    if (total > ncell_cap) return -1;
    for (int64_t i = 0; i < n; ++i) {
        int c3[3];
        for (int k = 0; k < 3; ++k) {
            double s = x[3 * i + k] / box[k];
            double w = s - floor(s);
            int c = (int)(w * (double)nc[k]);
            if (c >= nc[k]) c = nc[k] - 1;
            if (c < 0) c = 0;
            c3[k] = c;
        }
        cell_of[i] = c3[0] + nc[0] * (c3[1] + nc[1] * c3[2]);
    }
    for (long c = 0; c <= total; ++c) cell_start[c] = 0;
    for (int64_t i = 0; i < n; ++i) cell_start[cell_of[i] + 1] += 1;
    for (long c = 0; c < total; ++c) cell_start[c + 1] += cell_start[c];
    int32_t* fill = (int32_t*)malloc(sizeof(int32_t) * (size_t)(total > 0 ? total : 1));
    for (long c = 0; c < total; ++c) fill[c] = cell_start[c];
    for (int64_t i = 0; i < n; ++i) perm[fill[cell_of[i]]++] = (int32_t)i;  /* stable */
    free(fill);
    return (int)total;
}

/*
 * Uhlenbeck-Ford fluid (the liquid's reference system, Sec. 2.1 and Sec. 4):
 *   u(r) = -p kT ln(1 - exp(-r^2/sigma^2)) - u(rc)   for r < rc, else 0,
 * i.e. the UF pair potential with the energy scale p kT (kT fixed by the reference
 * temperature, not by the thermostat), truncated at rc and shifted there so that the energy
 * is continuous.  Force on j from i (d = x_j - x_i):  f_j = p kT (2/sigma^2) d / (exp(x) - 1)
 * with x = r^2/sigma^2 (repulsive).  Every unordered pair once, minimum image; box lengths
 * must exceed 2 rc.  Virial W_ab = sum over pairs d_a f_j,b.  Per-atom energy: half of each
 * pair term to each partner.  prm = [p, sigma, kT, rc].  Returns E, or NaN for a small box.
 */
double orc_uf_energy(int64_t n, const double* x, const double* box, const double* prm,
                     double* f, double* vir, double* eatom) {
    const double p = prm[0], sig = prm[1], kT = prm[2], rc = prm[3];
    for (int k = 0; k < 3; ++k) if (!(box[k] > 2.0 * rc)) return NAN;
    const double pk = p * kT, is2 = 1.0 / (sig * sig);
    const double shift = -pk * log(1.0 - exp(-rc * rc * is2));
    double E = 0.0, W[9] = {0};
    if (f) memset(f, 0, sizeof(double) * 3 * (size_t)n);
    if (eatom) memset(eatom, 0, sizeof(double) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t j = i + 1; j < n; ++j) {
            double d[3];
            for (int k = 0; k < 3; ++k) d[k] = min_image(x[3 * j + k], x[3 * i + k], box[k], NULL);
            double rr = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (!(rr < rc * rc)) continue;
            double xx = rr * is2;
            double u = -pk * log(1.0 - exp(-xx)) - shift;
            double c = 2.0 * pk * is2 / expm1(xx);   /* f_j = c d */
            E += u;
            if (eatom) { eatom[i] += 0.5 * u; eatom[j] += 0.5 * u; }
            if (f) for (int k = 0; k < 3; ++k) { f[3 * j + k] += c * d[k]; f[3 * i + k] -= c * d[k]; }
            for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) W[3 * a + b] += d[a] * c * d[b];
        }
    }
    if (vir) {
        vir[0] = W[0]; vir[1] = W[4]; vir[2] = W[8];
        vir[3] = W[1]; vir[4] = W[2]; vir[5] = W[5];
    }
    return E;
}
