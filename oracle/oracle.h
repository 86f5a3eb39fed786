/*
 * FP64 CPU oracle for the nucleon molecular-dynamics hot path of
 * Caplan, Schneider, Horowitz & Berry, "Pasta Nucleosynthesis: Molecular
 * dynamics simulations of nuclear statistical equilibrium" (arXiv:1412.8502).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the slow, obviously correct
 * reference that the CUDA path is checked against.  Only the test suite, the
 * smoke check and the CPU-baseline leg of the benchmark may load it; the
 * product library never links, calls or falls back to it.  It shares no code,
 * header, table or constant generator with the CUDA path.
 *
 * Everything is brute force: every pair of particles, nearest periodic image,
 * no cells, no lists, no blocking.  Arithmetic is IEEE FP64 compiled with
 * -ffp-contract=off.  Units: fm, MeV, fm/c (c = 1, k_B = 1).
 *
 * Layout: positions, velocities and forces are [N][3] row-major doubles
 * (particle-major).  type[i] = 1 for a proton, 0 for a neutron.
 *
 * Parity status: every function below is pinned by a CPU test against closed
 * forms, invariants or an independent brute-force implementation.  The
 * steepest-descent relaxation (orc_relax), whose constants are a reading of
 * the paper's "equilibrated from random" start, is pinned by one iteration
 * on two neutrons computed by hand from Table I (the clamp on the
 * displacement vector active and inactive) and by the energy decrease.
 */
#ifndef PASTA_ORACLE_H
#define PASTA_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    double a, b, c;      /* MeV, Table I */
    double Lambda;       /* fm^2, Table I */
    double lambda_s;     /* Coulomb screening length, fm (Sec. II.A: fixed at 10 fm) */
    double alpha;        /* alpha * hbar c, MeV fm */
    double M;            /* nucleon mass, MeV (Sec. II.A) */
    double r_nuc;        /* nuclear cutoff, fm (Sec. II.A: 11.5 fm) */
    double r_C;          /* Coulomb cutoff, fm (reading of Sec. II.A; <= L/2) */
    int coulomb;         /* 1: include the screened Coulomb term of V_pp */
} orc_params;

/* Table I and Sec. II.A defaults; r_C must be set by the caller. */
void orc_default_params(orc_params* p);

/* Eq. (1): pair potential between species ti, tj (1 = proton) at squared
 * separation r2.  Writes the nuclear and Coulomb parts of V and the scalar
 * g such that the force on i from j is g * (x_i - x_j).  Cutoffs are strict
 * (r2 < r_cut^2) and the truncated potential is not shifted. */
void orc_pair(int ti, int tj, double r2, const orc_params* p,
              double* v_nuc, double* v_coul, double* g);

/* Forces and energies by brute force over all pairs, nearest periodic image
 * (dx -= L * nearbyint(dx / L) per axis).  Targets i0 <= i < i1 get their
 * full force F[i] (rows outside the range are not touched); e_out (may be
 * NULL) receives, summed over those targets only,
 *   e_out[0] = 1/2 sum_i sum_{j!=i} V_nuc,  e_out[1] = same for V_coul,
 *   e_out[2] = 1/2 sum_i sum_{j!=i} (x_i - x_j).F_ij   (pair virial W),
 * so that for the full range they are sum_{i<j}.  Each per-target sum uses
 * Kahan compensation.  Runs OpenMP-parallel over targets. */
void orc_forces(int64_t N, const double* x, const int8_t* type, double L,
                const orc_params* p, int64_t i0, int64_t i1,
                double* F, double* e_out);

/* SplitMix64 (Steele, Lea & Flood 2014) k-th output of the stream that
 * starts at `seed` (k = 0 is the first call of next()). */
uint64_t orc_splitmix64(uint64_t seed, uint64_t k);

/* Initial state (reading of Sec. III.B "uniformly distributed random initial
 * positions"): N_p = floor(Yp*N + 0.5) protons first, L = cbrt(N/rho),
 * x[i][a] = U(3i+a) * L, Box-Muller Gaussians from draws 3N.. for the
 * velocities (sigma = sqrt(T/M)), centre-of-mass velocity removed, then an
 * exact rescale to KE = 3/2 N T.  U(k) = (splitmix64(seed,k) >> 11) * 2^-53.
 * Returns L. */
double orc_init(int64_t N, double Yp, double rho, double T, uint64_t seed,
                const orc_params* p, double* x, double* v, int8_t* type);

/* Steepest-descent relaxation used after orc_init: `iters` times
 * x += gamma*F with the per-particle displacement clamped to dmax, then
 * wrapped into [0, L). */
void orc_relax(int64_t N, double* x, const int8_t* type, double L,
               const orc_params* p, int64_t iters, double gamma, double dmax);

/* Wrap one coordinate into [0, L) (shared convention of the integrator). */
double orc_wrap(double x, double L);

typedef struct {
    double dt;             /* fm/c */
    double xi_dot;         /* expansion rate, c/fm (Eq. 3) */
    double L_base, t_base; /* L(t) = L_base * (1 + xi_dot * (t - t_base)) */
    double T;              /* thermostat temperature, MeV */
    int64_t thermostat_every; /* 0 = off; else rescale after every k-th step */
    int affine;            /* 1: scale positions by L_{n+1}/L_n after the box update
                              (an option outside the paper, which does not rescale) */
} orc_run_params;

/* Velocity Verlet with box expansion and isothermal rescale (Sec. II.A,
 * Eq. 3).  One step:
 *   v += dt/(2M) F;  x += dt v;  wrap x into [0, L);  F = F(x, L);
 *   v += dt/(2M) F;  t += dt;  step += 1;  L = L_base (1 + xi_dot (t - t_base));
 *   if thermostat_every > 0 and step % thermostat_every == 0:
 *       v *= sqrt(3/2 N T / KE).
 * F on entry must be F(x, L) for the entry state; it is updated in place.
 * t, step and L are in/out. */
void orc_run(int64_t N, double* x, double* v, double* F, const int8_t* type,
             const orc_params* p, const orc_run_params* rp, int64_t nsteps,
             double* t, int64_t* step, double* L);

/* Eq. (2): Thomas-Fermi screening length of a degenerate relativistic
 * electron gas of density n_e (fm^-3): lambda = sqrt(pi)/(2 sqrt(alpha))
 * (k_F sqrt(k_F^2 + m_e^2))^(-1/2), k_F = (3 pi^2 n_e)^(1/3), with the
 * fine-structure constant alpha and m_e in fm^-1 (hbar = c = 1). */
double orc_lambda_tf(double n_e);

/* Kinetic energy 1/2 M sum v^2 (Kahan). */
double orc_kinetic(int64_t N, const double* v, double M);

/* Cluster algorithm of Sec. II.C.  Protons linked when d^2 < r_pp^2 form
 * clusters (connected components); each cluster is labelled by its smallest
 * proton index.  A neutron joins the cluster of its nearest proton with
 * d^2 < r_np^2 (equal distances: the smaller proton index); otherwise it is
 * free (label -1).  d^2 uses the nearest periodic image in the form
 *   dx = x_i - x_j; if (dx > L/2) dx -= L; else if (dx < -L/2) dx += L;
 *   d2 = (dx*dx + dy*dy) + dz*dz       (no fused multiply-add)
 * hist_A[A] (size N+1) and hist_Z[Z] (size Np+1) count clusters by mass and
 * charge number.  stats[0] = number of clusters, stats[1] = free neutrons / N,
 * stats[2] = mean A and stats[3] = mean Z over clusters with A >= 12
 * (0 when there are none), stats[4] = number of clusters with A >= 12. */
void orc_clusters(int64_t N, const double* x, const int8_t* type, double L,
                  double r_pp, double r_np, int32_t* labels,
                  int64_t* hist_A, int64_t* hist_Z, double* stats);

/* MSTE clusters (energy criterion, a reading: the paper names the method in
 * Sec. II.C without defining it).  Nucleons i, j are bound when
 * V_ij(r) + (M/4)|v_i - v_j|^2 < 0 with V of Eq. (1) at the nearest image
 * (nuclear part inside r_nuc; Coulomb for proton pairs inside r_C, or always
 * with coulomb == 2); clusters are the connected components of bound pairs,
 * labelled by their smallest index; a neutron bound to nothing is free (-1),
 * a proton bound to nothing is its own cluster.  Outputs as orc_clusters.
 * v is [N][3] like x. */
void orc_mste(int64_t N, const double* x, const double* v, const int8_t* type, double L,
              const orc_params* p, int32_t* labels, int64_t* hist_A, int64_t* hist_Z, double* stats);

#ifdef __cplusplus
}
#endif
#endif
