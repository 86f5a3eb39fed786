/*
 * FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Plain definitions, brute force over all pairs, no cells, no lists.
 * Compiled with -O2 -fopenmp -ffp-contract=off.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* Table I (a, b, c, Lambda); Sec. II.A (M = 939 MeV, lambda = 10 fm,
 * r_nuc = 11.5 fm).  alpha in Eq. (1) multiplies 1/r, so dimensionally it is
 * the fine-structure constant times hbar*c (CODATA 2018 values). */
void orc_default_params(orc_params* p)
{
    p->a = 110.0;
    p->b = -26.0;
    p->c = 24.0;
    p->Lambda = 1.25;
    p->lambda_s = 10.0;
    p->alpha = 197.3269804 / 137.035999084;
    p->M = 939.0;
    p->r_nuc = 11.5;
    p->r_C = 0.0;
    p->coulomb = 1;
}

/* Eq. (1):
 *   V_np = a exp(-r^2/Lambda) + (b - c) exp(-r^2/(2 Lambda))
 *   V_nn = V_pp(nuclear) = a exp(-r^2/Lambda) + (b + c) exp(-r^2/(2 Lambda))
 *   V_pp adds alpha exp(-r/lambda) / r.
 * The force on i is -dV/dr * (x_i - x_j)/r, i.e. g * (x_i - x_j) with
 *   g = (2a/Lambda) e1 + ((b -+ c)/Lambda) e2
 *     + alpha exp(-r/lambda) (1/r^3 + 1/(lambda r^2)). */
void orc_pair(int ti, int tj, double r2, const orc_params* p,
              double* v_nuc, double* v_coul, double* g)
{
    double vn = 0.0, vc = 0.0, gg = 0.0;
    if (r2 < p->r_nuc * p->r_nuc) {
        double e1 = exp(-r2 / p->Lambda);
        double e2 = exp(-r2 / (2.0 * p->Lambda));
        double bc = (ti == tj) ? (p->b + p->c) : (p->b - p->c);
        vn = p->a * e1 + bc * e2;
        gg += (2.0 * p->a / p->Lambda) * e1 + (bc / p->Lambda) * e2;
    }
    if (ti == 1 && tj == 1 && p->coulomb && r2 < p->r_C * p->r_C) {
        double r = sqrt(r2);
        double ec = p->alpha * exp(-r / p->lambda_s);
        vc = ec / r;
        gg += ec * (1.0 / (r2 * r) + 1.0 / (p->lambda_s * r2));
    }
    *v_nuc = vn;
    *v_coul = vc;
    *g = gg;
}

static inline double min_image(double d, double L)
{
    return d - L * nearbyint(d / L);
}

typedef struct { double s, c; } kahan_t;

static inline void kahan_add(kahan_t* k, double v)
{
    double y = v - k->c;
    double t = k->s + y;
    k->c = (t - k->s) - y;
    k->s = t;
}

void orc_forces(int64_t N, const double* x, const int8_t* type, double L,
                const orc_params* p, int64_t i0, int64_t i1,
                double* F, double* e_out)
{
    int64_t n = i1 - i0;
    if (n <= 0) {
        if (e_out) e_out[0] = e_out[1] = e_out[2] = 0.0;
        return;
    }
    double* ep = (double*)calloc((size_t)n * 3, sizeof(double));

    #pragma omp parallel for schedule(dynamic, 8)
    for (int64_t i = i0; i < i1; ++i) {
        kahan_t fx = {0, 0}, fy = {0, 0}, fz = {0, 0};
        kahan_t en = {0, 0}, ec = {0, 0}, w = {0, 0};
        const double xi = x[3 * i], yi = x[3 * i + 1], zi = x[3 * i + 2];
        for (int64_t j = 0; j < N; ++j) {
            if (j == i) continue;
            double dx = min_image(xi - x[3 * j], L);
            double dy = min_image(yi - x[3 * j + 1], L);
            double dz = min_image(zi - x[3 * j + 2], L);
            double r2 = dx * dx + dy * dy + dz * dz;
            double vn, vc, g;
            orc_pair(type[i], type[j], r2, p, &vn, &vc, &g);
            if (g == 0.0 && vn == 0.0 && vc == 0.0) continue;
            kahan_add(&fx, g * dx);
            kahan_add(&fy, g * dy);
            kahan_add(&fz, g * dz);
            kahan_add(&en, vn);
            kahan_add(&ec, vc);
            kahan_add(&w, g * r2);
        }
        F[3 * i] = fx.s;
        F[3 * i + 1] = fy.s;
        F[3 * i + 2] = fz.s;
        ep[3 * (i - i0)] = 0.5 * en.s;
        ep[3 * (i - i0) + 1] = 0.5 * ec.s;
        ep[3 * (i - i0) + 2] = 0.5 * w.s;
    }
    if (e_out) {
        kahan_t a = {0, 0}, b = {0, 0}, c = {0, 0};
        for (int64_t k = 0; k < n; ++k) {
            kahan_add(&a, ep[3 * k]);
            kahan_add(&b, ep[3 * k + 1]);
            kahan_add(&c, ep[3 * k + 2]);
        }
        e_out[0] = a.s;
        e_out[1] = b.s;
        e_out[2] = c.s;
    }
    free(ep);
}

uint64_t orc_splitmix64(uint64_t seed, uint64_t k)
{
    /* next(): state += 0x9E3779B97F4A7C15; z = state; then the 64-bit
     * finaliser with shifts 30, 27, 31. */
    uint64_t z = seed + (k + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static inline double uniform01(uint64_t seed, uint64_t k)
{
    return (double)(orc_splitmix64(seed, k) >> 11) * 0x1.0p-53;
}

double orc_kinetic(int64_t N, const double* v, double M)
{
    kahan_t s = {0, 0};
    for (int64_t k = 0; k < 3 * N; ++k) kahan_add(&s, v[k] * v[k]);
    return 0.5 * M * s.s;
}

double orc_init(int64_t N, double Yp, double rho, double T, uint64_t seed,
                const orc_params* p, double* x, double* v, int8_t* type)
{
    double L = cbrt((double)N / rho);
    int64_t Np = (int64_t)floor(Yp * (double)N + 0.5);
    for (int64_t i = 0; i < N; ++i) type[i] = (i < Np) ? 1 : 0;
    for (int64_t k = 0; k < 3 * N; ++k) x[k] = uniform01(seed, (uint64_t)k) * L;

    double sigma = sqrt(T / p->M);
    const double two_pi = 6.283185307179586;
    for (int64_t k = 0; k < 3 * N; ++k) {
        int64_t m = k / 2;
        double u1 = uniform01(seed, (uint64_t)(3 * N + 2 * m));
        double u2 = uniform01(seed, (uint64_t)(3 * N + 2 * m + 1));
        double rad = sqrt(-2.0 * log(1.0 - u1));
        double ang = two_pi * u2;
        double g = (k % 2 == 0) ? rad * cos(ang) : rad * sin(ang);
        v[k] = sigma * g;
    }
    for (int a = 0; a < 3; ++a) {
        kahan_t s = {0, 0};
        for (int64_t i = 0; i < N; ++i) kahan_add(&s, v[3 * i + a]);
        double vcm = s.s / (double)N;
        for (int64_t i = 0; i < N; ++i) v[3 * i + a] -= vcm;
    }
    double ke = orc_kinetic(N, v, p->M);
    if (ke > 0.0) {
        double sc = sqrt(1.5 * (double)N * T / ke);
        for (int64_t k = 0; k < 3 * N; ++k) v[k] *= sc;
    } else {
        for (int64_t k = 0; k < 3 * N; ++k) v[k] = 0.0;
    }
    return L;
}

double orc_wrap(double x, double L)
{
    if (x >= L) {
        x -= L;
    } else if (x < 0.0) {
        x += L;
        if (x >= L) x = 0.0;
    }
    return x;
}

void orc_relax(int64_t N, double* x, const int8_t* type, double L,
               const orc_params* p, int64_t iters, double gamma, double dmax)
{
    double* F = (double*)malloc((size_t)N * 3 * sizeof(double));
    for (int64_t it = 0; it < iters; ++it) {
        orc_forces(N, x, type, L, p, 0, N, F, NULL);
        for (int64_t i = 0; i < N; ++i) {
            double d0 = gamma * F[3 * i], d1 = gamma * F[3 * i + 1], d2 = gamma * F[3 * i + 2];
            double m = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
            if (m > dmax) {
                double s = dmax / m;
                d0 *= s;
                d1 *= s;
                d2 *= s;
            }
            x[3 * i] = orc_wrap(x[3 * i] + d0, L);
            x[3 * i + 1] = orc_wrap(x[3 * i + 1] + d1, L);
            x[3 * i + 2] = orc_wrap(x[3 * i + 2] + d2, L);
        }
    }
    free(F);
}

void orc_run(int64_t N, double* x, double* v, double* F, const int8_t* type,
             const orc_params* p, const orc_run_params* rp, int64_t nsteps,
             double* t, int64_t* step, double* L)
{
    const double h = 0.5 * rp->dt / p->M;
    for (int64_t s = 0; s < nsteps; ++s) {
        for (int64_t k = 0; k < 3 * N; ++k) v[k] += h * F[k];
        for (int64_t k = 0; k < 3 * N; ++k) x[k] = orc_wrap(x[k] + rp->dt * v[k], *L);
        orc_forces(N, x, type, *L, p, 0, N, F, NULL);
        for (int64_t k = 0; k < 3 * N; ++k) v[k] += h * F[k];
        *t += rp->dt;
        *step += 1;
        const double L_old = *L;
        *L = rp->L_base * (1.0 + rp->xi_dot * (*t - rp->t_base));
        if (rp->affine) {
            const double sc = *L / L_old;
            for (int64_t k = 0; k < 3 * N; ++k) x[k] *= sc;
        }
        if (rp->thermostat_every > 0 && (*step % rp->thermostat_every) == 0) {
            double ke = orc_kinetic(N, v, p->M);
            if (ke > 0.0) {
                double sc = sqrt(1.5 * (double)N * rp->T / ke);
                for (int64_t k = 0; k < 3 * N; ++k) v[k] *= sc;
            }
        }
    }
}

double orc_lambda_tf(double n_e)
{
    const double pi = 3.14159265358979323846;
    const double alpha = 1.0 / 137.035999084;
    const double me = 0.51099895 / 197.3269804;     /* electron mass, fm^-1 */
    const double kF = cbrt(3.0 * pi * pi * n_e);
    return sqrt(pi) / (2.0 * sqrt(alpha)) / sqrt(kF * sqrt(kF * kF + me * me));
}

static int64_t uf_find(int64_t* parent, int64_t a)
{
    while (parent[a] != a) {
        parent[a] = parent[parent[a]];
        a = parent[a];
    }
    return a;
}

static inline double cl_d2(const double* xi, const double* xj, double L)
{
    double h = 0.5 * L;
    double d[3];
    for (int a = 0; a < 3; ++a) {
        double dx = xi[a] - xj[a];
        if (dx > h) dx -= L;
        else if (dx < -h) dx += L;
        d[a] = dx;
    }
    double s = d[0] * d[0];
    s = s + d[1] * d[1];
    s = s + d[2] * d[2];
    return s;
}

void orc_clusters(int64_t N, const double* x, const int8_t* type, double L,
                  double r_pp, double r_np, int32_t* labels,
                  int64_t* hist_A, int64_t* hist_Z, double* stats)
{
    /* Protons, in index order. */
    int64_t Np = 0;
    for (int64_t i = 0; i < N; ++i) Np += (type[i] == 1);
    int64_t* pidx = (int64_t*)malloc((size_t)(Np > 0 ? Np : 1) * sizeof(int64_t));
    int64_t* parent = (int64_t*)malloc((size_t)(Np > 0 ? Np : 1) * sizeof(int64_t));
    int64_t k = 0;
    for (int64_t i = 0; i < N; ++i)
        if (type[i] == 1) pidx[k++] = i;
    for (int64_t a = 0; a < Np; ++a) parent[a] = a;

    const double rpp2 = r_pp * r_pp, rnp2 = r_np * r_np;
    /* The edges (proton pairs closer than r_pp) are found by all threads,
     * each proton a testing every b > a into a buffer of its thread; the
     * clusters are the connected components of these edges, joined
     * afterwards in one thread (the components do not depend on the order
     * the edges are joined in). */
    int64_t* edges = NULL;
    int64_t nedges = 0;
    #pragma omp parallel
    {
        int64_t* buf = NULL;
        int64_t n = 0, cap = 0;
        #pragma omp for schedule(dynamic, 64)
        for (int64_t a = 0; a < Np; ++a)
            for (int64_t b = a + 1; b < Np; ++b)
                if (cl_d2(&x[3 * pidx[a]], &x[3 * pidx[b]], L) < rpp2) {
                    if (n == cap) {
                        cap = cap ? 2 * cap : 1024;
                        buf = (int64_t*)realloc(buf, (size_t)(2 * cap) * sizeof(int64_t));
                    }
                    buf[2 * n] = a;
                    buf[2 * n + 1] = b;
                    n++;
                }
        #pragma omp critical
        {
            edges = (int64_t*)realloc(edges, (size_t)(2 * (nedges + n) + 2) * sizeof(int64_t));
            if (n) memcpy(edges + 2 * nedges, buf, (size_t)(2 * n) * sizeof(int64_t));
            nedges += n;
        }
        free(buf);
    }
    for (int64_t e = 0; e < nedges; ++e) {
        int64_t ra = uf_find(parent, edges[2 * e]), rb = uf_find(parent, edges[2 * e + 1]);
        if (ra != rb) {
            if (ra < rb) parent[rb] = ra;
            else parent[ra] = rb;
        }
    }
    free(edges);
    /* The root of each component is its smallest member because roots only
     * ever point to smaller roots. */
    for (int64_t i = 0; i < N; ++i) labels[i] = -1;
    for (int64_t a = 0; a < Np; ++a) labels[pidx[a]] = (int32_t)pidx[uf_find(parent, a)];

    /* each neutron independently (labels of protons are final here) */
    #pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < N; ++i) {
        if (type[i] == 1) continue;
        int64_t best = -1;
        double bestd2 = 0.0;
        for (int64_t a = 0; a < Np; ++a) {
            double d2 = cl_d2(&x[3 * i], &x[3 * pidx[a]], L);
            if (d2 < rnp2 && (best < 0 || d2 < bestd2)) {
                best = a;
                bestd2 = d2;
            }
        }
        labels[i] = (best < 0) ? -1 : labels[pidx[best]];
    }

    int64_t* zc = (int64_t*)calloc((size_t)(N > 0 ? N : 1), sizeof(int64_t));
    int64_t* ac = (int64_t*)calloc((size_t)(N > 0 ? N : 1), sizeof(int64_t));
    int64_t nfree = 0;
    for (int64_t i = 0; i < N; ++i) {
        if (labels[i] < 0) { nfree++; continue; }
        ac[labels[i]] += 1;
        if (type[i] == 1) zc[labels[i]] += 1;
    }
    memset(hist_A, 0, (size_t)(N + 1) * sizeof(int64_t));
    memset(hist_Z, 0, (size_t)(Np + 1) * sizeof(int64_t));
    int64_t ncl = 0, nbig = 0, sumA = 0, sumZ = 0;
    for (int64_t i = 0; i < N; ++i) {
        if (type[i] == 1 && labels[i] == (int32_t)i) {
            ncl++;
            hist_A[ac[i]] += 1;
            hist_Z[zc[i]] += 1;
            if (ac[i] >= 12) {
                nbig++;
                sumA += ac[i];
                sumZ += zc[i];
            }
        }
    }
    stats[0] = (double)ncl;
    stats[1] = (double)nfree / (double)N;
    stats[2] = nbig ? (double)sumA / (double)nbig : 0.0;
    stats[3] = nbig ? (double)sumZ / (double)nbig : 0.0;
    stats[4] = (double)nbig;
    free(zc);
    free(ac);
    free(pidx);
    free(parent);
}

/* ------------------------------------------------------------------------
 * Minimum spanning tree in two-particle energy space (MSTE), the
 * energy-based cluster criterion the paper names beside its distance
 * algorithm (Sec. II.C).  Reading: nucleons i and j are bound when
 *   e_ij = V_ij(r_ij) + (M/4) |v_i - v_j|^2 < 0,
 * V_ij the pair potential of Eq. (1) (nuclear part for r < r_nuc; screened
 * Coulomb for proton pairs, inside r_C when coulomb == 1, always when
 * coulomb == 2) at the nearest image, (M/4)|dv|^2 the kinetic energy of the
 * relative motion (reduced mass M/2).  Clusters are the connected
 * components of the bound pairs (the components of a minimum spanning tree
 * over the negative-energy edges).  Pairs at r >= r_nuc have V >= 0 and are
 * never bound.  Every operation below is one IEEE FP64 operation in this
 * order (no contraction):
 *   d = x_i - x_j per axis, nearest image by comparison with L/2;
 *   r2 = (dx*dx + dy*dy) + dz*dz;  g = exp(-r2 / (2 Lambda));
 *   V = ((a*g)*g + s*g) + [pp] (alpha*exp(-sqrt(r2)/lambda)) / sqrt(r2);
 *   k = (dvx*dvx + dvy*dvy) + dvz*dvz;  e = V + (M/4)*k.
 * Labels: the smallest index of the component; a neutron bound to nothing
 * is free (-1); a proton bound to nothing is a cluster by itself (as in
 * Sec. II.C).  hist_A / hist_Z / stats as in orc_clusters (clusters of
 * neutrons only count in hist_Z[0]).
 * ---------------------------------------------------------------------- */
static double ms_pair_energy(const double* xi, const double* xj, const double* vi, const double* vj,
                             int ti, int tj, double L, const orc_params* p, int* in_range)
{
    const double r2 = cl_d2(xi, xj, L);
    *in_range = r2 < p->r_nuc * p->r_nuc;
    if (!*in_range) return 0.0;
    const double s = (ti == tj) ? (p->b + p->c) : (p->b - p->c);
    const double g = exp(-r2 / (2.0 * p->Lambda));
    double v = (p->a * g) * g + s * g;
    if (ti == 1 && tj == 1 && p->coulomb && (p->coulomb == 2 || r2 < p->r_C * p->r_C)) {
        const double r = sqrt(r2);
        v = v + (p->alpha * exp(-r / p->lambda_s)) / r;
    }
    const double dx = vi[0] - vj[0], dy = vi[1] - vj[1], dz = vi[2] - vj[2];
    const double k = (dx * dx + dy * dy) + dz * dz;
    return v + (0.25 * p->M) * k;
}

void orc_mste(int64_t N, const double* x, const double* v, const int8_t* type, double L,
              const orc_params* p, int32_t* labels, int64_t* hist_A, int64_t* hist_Z, double* stats)
{
    int64_t* parent = (int64_t*)malloc((size_t)(N > 0 ? N : 1) * sizeof(int64_t));
    int64_t* deg = (int64_t*)calloc((size_t)(N > 0 ? N : 1), sizeof(int64_t));
    int64_t Np = 0;
    for (int64_t i = 0; i < N; ++i) {
        parent[i] = i;
        Np += (type[i] == 1);
    }
    for (int64_t i = 0; i < N; ++i)
        for (int64_t j = i + 1; j < N; ++j) {
            int in = 0;
            const double e = ms_pair_energy(&x[3 * i], &x[3 * j], &v[3 * i], &v[3 * j], type[i], type[j], L, p, &in);
            if (in && e < 0.0) {
                deg[i]++;
                deg[j]++;
                int64_t ri = uf_find(parent, i), rj = uf_find(parent, j);
                if (ri != rj) {
                    if (ri < rj) parent[rj] = ri;
                    else parent[ri] = rj;
                }
            }
        }
    for (int64_t i = 0; i < N; ++i)
        labels[i] = (type[i] == 0 && deg[i] == 0) ? -1 : (int32_t)uf_find(parent, i);

    int64_t* zc = (int64_t*)calloc((size_t)(N > 0 ? N : 1), sizeof(int64_t));
    int64_t* ac = (int64_t*)calloc((size_t)(N > 0 ? N : 1), sizeof(int64_t));
    int64_t nfree = 0;
    for (int64_t i = 0; i < N; ++i) {
        if (labels[i] < 0) { nfree++; continue; }
        ac[labels[i]] += 1;
        if (type[i] == 1) zc[labels[i]] += 1;
    }
    memset(hist_A, 0, (size_t)(N + 1) * sizeof(int64_t));
    memset(hist_Z, 0, (size_t)(Np + 1) * sizeof(int64_t));
    int64_t ncl = 0, nbig = 0, sumA = 0, sumZ = 0;
    for (int64_t i = 0; i < N; ++i) {
        if (labels[i] == (int32_t)i) {
            ncl++;
            hist_A[ac[i]] += 1;
            hist_Z[zc[i]] += 1;
            if (ac[i] >= 12) {
                nbig++;
                sumA += ac[i];
                sumZ += zc[i];
            }
        }
    }
    stats[0] = (double)ncl;
    stats[1] = (double)nfree / (double)N;
    stats[2] = nbig ? (double)sumA / (double)nbig : 0.0;
    stats[3] = nbig ? (double)sumZ / (double)nbig : 0.0;
    stats[4] = (double)nbig;
    free(zc);
    free(ac);
    free(deg);
    free(parent);
}
