/*
 * Plain FP64 CPU oracle for short-range pair forces and velocity Verlet.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only tests/, __graft_entry__.smoke() and bench.py's CPU
 * baseline leg use it.  It shares no code, header, table or constant with the
 * CUDA library; it is the slow, obviously correct statement of what that
 * library computes, so a reader can check it against the paper by eye.
 *
 * Sources (Vance et al., "Code modernization strategies for short-range
 * non-bonded molecular dynamics simulations", arXiv:2109.10876):
 *   - Newton's equations m_i r_i'' = F_i, F = -grad U            (Eq. 1, Sec. 2.1)
 *   - Lennard-Jones V(r) = 4 eps [(sigma/r)^12 - (sigma/r)^6],
 *     interactions restricted to r < r_cut                         (Eq. 2, Sec. 2.1.1)
 *   - repulsive LJ (WCA) with r_cut = 2^(1/6) sigma                (Sec. 4, polymer melt)
 *   - Verlet list = pairs within r_cut + r_skin                     (Sec. 2.1.2)
 *   - velocity Verlet in two half steps (Integrate1 / Integrate2)   (Fig. 1, Sec. 2.1)
 *   - FENE bonds along chains, Langevin thermostat                  (Sec. 4)
 *
 * Readings where the paper is silent:
 *   - the LJ energy is shifted so that V_s(r_cut) = 0 (forces unchanged);
 *     WCA is the same shifted form with r_cut = 2^(1/6) sigma, i.e. V + eps;
 *   - the Langevin thermostat is a force term -gamma m v + sqrt(24 gamma kT m/dt) u,
 *     u uniform in (-1/2, 1/2) from Philox4x32-10 keyed by (seed) and counted by
 *     (particle id, step), applied with the velocity available at force time;
 *   - minimum image d -= L * nearbyint(d / L) per axis (valid for L >= 2 r_cut);
 *   - the angle term on triples along a chain (Sec. 4 names a cosine-type
 *     term on triples without its form) is U = K (1 - cos theta), theta
 *     the angle between consecutive bond vectors b1 = x_b - x_a and
 *     b2 = x_c - x_b (0 for a straight chain);
 *   - the soft push-off used to prepare overlapping polymer chains before the
 *     WCA melt run (Sec. 4 names the melt, not its preparation) is the cosine
 *     potential V = A (1 + cos(pi r / r_cut)) for r < r_cut, with A = eps.
 *
 * Layout: positions, velocities and forces are row-major N x 3 arrays
 * (x0, y0, z0, x1, ...).  All arithmetic is IEEE FP64; build with
 * -ffp-contract=off so that every product and sum is rounded separately,
 * which makes the squared distance below a fixed, reproducible function of
 * the two positions.
 */
#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* System description (plain struct, mirrored by oracle/__init__.py)    */
/* ------------------------------------------------------------------ */
typedef struct {
    int64_t n;            /* number of particles                         */
    double box[3];        /* orthorhombic periodic box (Lx, Ly, Lz)      */
    double eps, sigma;    /* LJ parameters (Eq. 2)                       */
    double rc;            /* cutoff radius (absolute, not in sigma)      */
    int32_t shift;        /* 1: subtract V(rc) from the pair energy      */
    double mass;          /* particle mass (reduced units: 1)            */
    double dt;            /* time step                                   */
    double gamma, kT;     /* Langevin friction and temperature; gamma=0 -> NVE */
    uint64_t seed;        /* Philox key                                  */
    int64_t n_bonds;      /* FENE bonds                                  */
    const int32_t *bonds; /* 2*n_bonds particle ids, or NULL             */
    double fene_K, fene_R0;
    int32_t pot;          /* 0: LJ / WCA (Eq. 2), 1: soft cosine push-off  */
    double angle_K;       /* bending constant of the angle term           */
    int64_t n_angles;     /* angle triples (a, b, c), b the middle bead   */
    const int32_t *angles;/* 3*n_angles particle ids, or NULL             */
} orc_system;

enum { ORC_OK = 0, ORC_ERR_BOND = -5, ORC_ERR_CAP = -3, ORC_ERR_ARG = -1 };

/* ------------------------------------------------------------------ */
/* Pair potential (Eq. 2)                                              */
/* ------------------------------------------------------------------ */

/* Unshifted LJ energy at distance r. */
double orc_lj_energy(double r, double eps, double sigma)
{
    double sr = sigma / r;
    double sr6 = sr * sr * sr * sr * sr * sr;
    return 4.0 * eps * (sr6 * sr6 - sr6);
}

/* Magnitude of the pair force along the separation, -dV/dr, at distance r.
 * dV/dr = 4 eps [-12 sigma^12 / r^13 + 6 sigma^6 / r^7]. */
double orc_lj_force(double r, double eps, double sigma)
{
    double sr = sigma / r;
    double sr6 = sr * sr * sr * sr * sr * sr;
    return 24.0 * eps * (2.0 * sr6 * sr6 - sr6) / r;
}

/* Minimum-image separation d = x_i - x_j in an orthorhombic periodic box,
 * and its squared length.  The sequence of roundings is fixed:
 * d_k = x_ik - x_jk; d_k = d_k - L_k * nearbyint(d_k / L_k);
 * r2 = (dx*dx + dy*dy) + dz*dz. */
static double min_image(const double *xi, const double *xj, const double *L, double d[3])
{
    for (int k = 0; k < 3; ++k) {
        double t = xi[k] - xj[k];
        double q = nearbyint(t / L[k]);
        double s = L[k] * q;
        d[k] = t - s;
    }
    double a = d[0] * d[0];
    double b = d[1] * d[1];
    double c = d[2] * d[2];
    return (a + b) + c;
}

double orc_min_image_r2(const double *xi, const double *xj, const double *box)
{
    double d[3];
    return min_image(xi, xj, box, d);
}

/* Soft cosine push-off V(r) = A (1 + cos(pi r / rc)) for r < rc: V(0) = 2A,
 * V(rc) = 0 and dV/dr(rc) = 0.  Its force -dV/dr = (pi A / rc) sin(pi r / rc)
 * is bounded by pi A / rc, so fully overlapping beads can be separated. */
double orc_soft_energy(double r, double A, double rc)
{
    return A * (1.0 + cos(M_PI * r / rc));
}

double orc_soft_force(double r, double A, double rc)
{
    return M_PI * A / rc * sin(M_PI * r / rc);
}

/* Pair force on i from j and pair energy for separation d (r2 = |d|^2 < rc^2). */
static void lj_pair(const orc_system *s, const double d[3], double r2,
                    double f[3], double *v_pair, double *w_pair)
{
    if (s->pot == 1) {
        double r = sqrt(r2);
        double fmag = orc_soft_force(r, s->eps, s->rc);
        /* coincident particles: V = 2A, no direction, no force */
        for (int k = 0; k < 3; ++k) f[k] = r > 0.0 ? fmag * d[k] / r : 0.0;
        *v_pair = orc_soft_energy(r, s->eps, s->rc);
        *w_pair = d[0] * f[0] + d[1] * f[1] + d[2] * f[2];
        return;
    }
    double r = sqrt(r2);
    double fmag = orc_lj_force(r, s->eps, s->sigma);  /* -dV/dr */
    double v = orc_lj_energy(r, s->eps, s->sigma);
    if (s->shift) v -= orc_lj_energy(s->rc, s->eps, s->sigma);
    /* V depends on r = |x_i - x_j|, so F_i = -dV/dx_i = (-dV/dr) d / r. */
    for (int k = 0; k < 3; ++k) f[k] = fmag * d[k] / r;
    *v_pair = v;
    *w_pair = d[0] * f[0] + d[1] * f[1] + d[2] * f[2];
}

/* ------------------------------------------------------------------ */
/* FENE bond (Kremer-Grest, cited in Sec. 4)                          */
/* U = -1/2 K R0^2 ln(1 - r^2/R0^2), F_i = -K d / (1 - r^2/R0^2)       */
/* ------------------------------------------------------------------ */
static int fene_pair(const orc_system *s, const double d[3], double r2,
                     double f[3], double *u, double *w)
{
    double R02 = s->fene_R0 * s->fene_R0;
    double q = 1.0 - r2 / R02;
    if (!(q > 0.0)) return ORC_ERR_BOND;
    double c = -s->fene_K / q;
    for (int k = 0; k < 3; ++k) f[k] = c * d[k];
    *u = -0.5 * s->fene_K * R02 * log(q);
    *w = d[0] * f[0] + d[1] * f[1] + d[2] * f[2];
    return ORC_OK;
}

/* Cosine angle term U = K (1 - cos theta) of one triple (a, b, c) with bond
 * vectors b1 = x_b - x_a, b2 = x_c - x_b (minimum image), c = b1.b2/(l1 l2):
 * F_a = -K (b2/(l1 l2) - c b1/l1^2), F_c = K (b1/(l1 l2) - c b2/l2^2),
 * F_b = -(F_a + F_c).  U depends only on the angle, so its virial is zero. */
double orc_angle_energy(const double b1[3], const double b2[3], double K)
{
    double l1 = sqrt(b1[0] * b1[0] + b1[1] * b1[1] + b1[2] * b1[2]);
    double l2 = sqrt(b2[0] * b2[0] + b2[1] * b2[1] + b2[2] * b2[2]);
    double c = (b1[0] * b2[0] + b1[1] * b2[1] + b1[2] * b2[2]) / (l1 * l2);
    return K * (1.0 - c);
}

static void angle_forces(const double b1[3], const double b2[3], double K,
                         double fa[3], double fb[3], double fc[3])
{
    double l1s = b1[0] * b1[0] + b1[1] * b1[1] + b1[2] * b1[2];
    double l2s = b2[0] * b2[0] + b2[1] * b2[1] + b2[2] * b2[2];
    double l12 = sqrt(l1s) * sqrt(l2s);
    double c = (b1[0] * b2[0] + b1[1] * b2[1] + b1[2] * b2[2]) / l12;
    for (int k = 0; k < 3; ++k) {
        fa[k] = -K * (b2[k] / l12 - c * b1[k] / l1s);
        fc[k] = K * (b1[k] / l12 - c * b2[k] / l2s);
        fb[k] = -(fa[k] + fc[k]);
    }
}

/* Forces of the triple (a, b, c) at positions x (box L): fa, fb, fc and U. */
void orc_angle_triple(const double *xa, const double *xb, const double *xc, const double *box, double K,
                      double *fa, double *fb, double *fc, double *u)
{
    double b1[3], b2[3];
    min_image(xb, xa, box, b1);
    min_image(xc, xb, box, b2);
    angle_forces(b1, b2, K, fa, fb, fc);
    *u = orc_angle_energy(b1, b2, K);
}

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), from its          */
/* published definition: 10 rounds of two 32x32->64 multiplies, with    */
/* the key bumped by the Weyl constants between rounds.                 */
/* ------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        if (round < 9) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform variate in (-1/2, 1/2) from one 32-bit word; exact in FP64. */
static double u_centered(uint32_t r)
{
    return ((double)r + 0.5) * (1.0 / 4294967296.0) - 0.5;
}

/* Langevin noise for particle id at step: three uniforms in (-1/2, 1/2). */
void orc_langevin_uniforms(uint64_t seed, int64_t id, int64_t step, double u[3])
{
    uint32_t ctr[4] = { (uint32_t)id, (uint32_t)(uint64_t)step,
                        (uint32_t)((uint64_t)step >> 32), 0x4C414E47u };
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    uint32_t r[4];
    orc_philox4x32_10(ctr, key, r);
    for (int k = 0; k < 3; ++k) u[k] = u_centered(r[k]);
}

/* ------------------------------------------------------------------ */
/* Forces: direct O(N^2) sum over all j != i, minimum image           */
/* ------------------------------------------------------------------ */

/* Pair force on particle i (non-bonded only) and its half of the pair
 * energy and virial (each pair is visited from both ends). */
static void pair_row(const orc_system *s, const double *x, int64_t i,
                     double Fi[3], double *Ui, double *Wi)
{
    double rc2 = s->rc * s->rc;
    double F[3] = {0, 0, 0}, U = 0, W = 0;
    for (int64_t j = 0; j < s->n; ++j) {
        if (j == i) continue;
        double d[3];
        double r2 = min_image(&x[3 * i], &x[3 * j], s->box, d);
        if (r2 < rc2) {                 /* strict r < r_cut (Eq. 2 text) */
            double f[3], v, w;
            lj_pair(s, d, r2, f, &v, &w);
            for (int k = 0; k < 3; ++k) F[k] += f[k];
            U += 0.5 * v;
            W += 0.5 * w;
        }
    }
    for (int k = 0; k < 3; ++k) Fi[k] = F[k];
    *Ui = U;
    *Wi = W;
}

/* Total conservative force (LJ/WCA + FENE) on every particle; euw gets
 * (U, K, W): potential energy, kinetic energy 1/2 m sum v^2 (v may be NULL,
 * then K = 0) and the virial sum over pairs of d_ij . f_ij.
 * Per-particle energies (U_i, W_i halves) go to ui/wi if non-NULL. */
int orc_forces(const orc_system *s, const double *x, const double *v,
               double *F, double *euw)
{
    int64_t n = s->n;
    double U = 0, W = 0, K = 0;
    double *Urow = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *Wrow = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!Urow || !Wrow) { free(Urow); free(Wrow); return ORC_ERR_ARG; }
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) pair_row(s, x, i, &F[3 * i], &Urow[i], &Wrow[i]);
    for (int64_t i = 0; i < n; ++i) { U += Urow[i]; W += Wrow[i]; }
    free(Urow);
    free(Wrow);
    int rc = ORC_OK;
    for (int64_t b = 0; b < s->n_bonds && s->bonds; ++b) {
        int64_t i = s->bonds[2 * b], j = s->bonds[2 * b + 1];
        double d[3], f[3], u, w;
        double r2 = min_image(&x[3 * i], &x[3 * j], s->box, d);
        if (fene_pair(s, d, r2, f, &u, &w) != ORC_OK) { rc = ORC_ERR_BOND; continue; }
        for (int k = 0; k < 3; ++k) { F[3 * i + k] += f[k]; F[3 * j + k] -= f[k]; }
        U += u;
        W += w;
    }
    for (int64_t t = 0; t < s->n_angles && s->angles; ++t) {
        int64_t a = s->angles[3 * t], b = s->angles[3 * t + 1], c = s->angles[3 * t + 2];
        double fa[3], fb[3], fc[3], u;
        orc_angle_triple(&x[3 * a], &x[3 * b], &x[3 * c], s->box, s->angle_K, fa, fb, fc, &u);
        for (int k = 0; k < 3; ++k) { F[3 * a + k] += fa[k]; F[3 * b + k] += fb[k]; F[3 * c + k] += fc[k]; }
        U += u;
    }
    if (v) for (int64_t i = 0; i < n; ++i)
        K += 0.5 * s->mass * (v[3 * i] * v[3 * i] + v[3 * i + 1] * v[3 * i + 1] + v[3 * i + 2] * v[3 * i + 2]);
    if (euw) { euw[0] = U; euw[1] = K; euw[2] = W; }
    return rc;
}

/* Non-bonded forces on a chosen subset of particles (exact for those
 * particles: each sums over all j), for systems too large for the full
 * O(N^2) sum.  Fs is n_sample x 3, ui/wi per sampled particle may be NULL. */
int orc_forces_sample(const orc_system *s, const double *x, int64_t n_sample,
                      const int64_t *idx, double *Fs, double *ui, double *wi)
{
    for (int64_t q = 0; q < n_sample; ++q)
        if (idx[q] < 0 || idx[q] >= s->n) return ORC_ERR_ARG;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t q = 0; q < n_sample; ++q) {
        double U, W;
        pair_row(s, x, idx[q], &Fs[3 * q], &U, &W);
        if (ui) ui[q] = U;
        if (wi) wi[q] = W;
    }
    return ORC_OK;
}

/* Bonded forces (FENE bonds and angle triples, Sec. 4) on chosen particles: */
/* for each sample, the bonds and triples it belongs to are found by a scan  */
/* of the whole bond and triple lists, and their forces on it summed.  The   */
/* counterpart of orc_forces_sample for the bonded terms; Fs is n_sample x 3. */
int orc_bonded_sample(const orc_system *s, const double *x, int64_t n_sample,
                      const int64_t *idx, double *Fs)
{
    for (int64_t q = 0; q < n_sample; ++q)
        if (idx[q] < 0 || idx[q] >= s->n) return ORC_ERR_ARG;
    int rc = ORC_OK;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t q = 0; q < n_sample; ++q) {
        const int64_t i = idx[q];
        double F[3] = {0, 0, 0};
        for (int64_t b = 0; b < s->n_bonds && s->bonds; ++b) {
            const int64_t a = s->bonds[2 * b], c = s->bonds[2 * b + 1];
            if (a != i && c != i) continue;
            const int64_t j = (a == i) ? c : a;
            double d[3], f[3], u, w;
            const double r2 = min_image(&x[3 * i], &x[3 * j], s->box, d);
            if (fene_pair(s, d, r2, f, &u, &w) != ORC_OK) {
#pragma omp atomic write
                rc = ORC_ERR_BOND;
                continue;
            }
            for (int k = 0; k < 3; ++k) F[k] += f[k];
        }
        for (int64_t t = 0; t < s->n_angles && s->angles; ++t) {
            const int64_t a = s->angles[3 * t], b = s->angles[3 * t + 1], c = s->angles[3 * t + 2];
            if (a != i && b != i && c != i) continue;
            double fa[3], fb[3], fc[3], u;
            orc_angle_triple(&x[3 * a], &x[3 * b], &x[3 * c], s->box, s->angle_K, fa, fb, fc, &u);
            const double *f = (a == i) ? fa : (b == i ? fb : fc);
            for (int k = 0; k < 3; ++k) F[k] += f[k];
        }
        for (int k = 0; k < 3; ++k) Fs[3 * q + k] = F[k];
    }
    return rc;
}

/* Langevin force on particle i at a given step, using velocity vi. */
static void langevin_force(const orc_system *s, int64_t i, int64_t step, const double *vi, double f[3])
{
    double u[3];
    orc_langevin_uniforms(s->seed, i, step, u);
    double amp = sqrt(24.0 * s->gamma * s->kT * s->mass / s->dt);
    for (int k = 0; k < 3; ++k) f[k] = -s->gamma * s->mass * vi[k] + amp * u[k];
}

/* The Langevin force of chosen particles at a given step, with their       */
/* velocities vs (n_sample x 3) as the integrator would use them.            */
void orc_langevin_sample(const orc_system *s, int64_t n_sample, const int64_t *idx, const double *vs,
                         int64_t step, double *Fs)
{
    for (int64_t q = 0; q < n_sample; ++q) langevin_force(s, idx[q], step, &vs[3 * q], &Fs[3 * q]);
}

/* Total force used by the integrator: conservative + (if gamma > 0) Langevin. */
static int total_force(const orc_system *s, const double *x, const double *v,
                       int64_t step, double *F, double *euw)
{
    int rc = orc_forces(s, x, v, F, euw);
    if (s->gamma > 0.0) {
        for (int64_t i = 0; i < s->n; ++i) {
            double f[3];
            langevin_force(s, i, step, &v[3 * i], f);
            for (int k = 0; k < 3; ++k) F[3 * i + k] += f[k];
        }
    }
    return rc;
}

/* Wrap a coordinate into [0, L). */
static double wrap(double y, double L)
{
    if (y >= L) y = y - L;
    if (y < 0.0) {
        y = y + L;
        if (y >= L) y = 0.0;
    }
    return y;
}

/* ------------------------------------------------------------------ */
/* Velocity Verlet (Fig. 1): Integrate1 = half kick + drift,           */
/* force evaluation, Integrate2 = half kick.                           */
/* ------------------------------------------------------------------ */
/* Runs nsteps steps starting at step counter step0 from (x, v); the force at
 * the start is evaluated with the current v (Langevin) and counter step0.
 * On return x, v hold the state after nsteps, F the force at the final x.
 * thermo (may be NULL) receives 3*nsteps values (U, K, W) after each step,
 * K evaluated with the synchronised velocity at the end of the step. */
int orc_vv_run(const orc_system *s, double *x, double *v, double *F,
               int64_t step0, int64_t nsteps, double *thermo)
{
    int64_t n = s->n;
    double h = 0.5 * s->dt / s->mass;
    int rc = total_force(s, x, v, step0, F, NULL);
    if (rc != ORC_OK) return rc;
    for (int64_t t = 1; t <= nsteps; ++t) {
        for (int64_t i = 0; i < n; ++i)
            for (int k = 0; k < 3; ++k) {
                v[3 * i + k] += h * F[3 * i + k];
                x[3 * i + k] = wrap(x[3 * i + k] + s->dt * v[3 * i + k], s->box[k]);
            }
        double euw[3];
        rc = total_force(s, x, v, step0 + t, F, euw);
        if (rc != ORC_OK) return rc;
        double K = 0.0;
        for (int64_t i = 0; i < n; ++i)
            for (int k = 0; k < 3; ++k) {
                v[3 * i + k] += h * F[3 * i + k];
                K += 0.5 * s->mass * v[3 * i + k] * v[3 * i + k];
            }
        if (thermo) {
            thermo[3 * (t - 1) + 0] = euw[0];
            thermo[3 * (t - 1) + 1] = K;
            thermo[3 * (t - 1) + 2] = euw[2];
        }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Verlet pair set (Sec. 2.1.2): all i < j with |d_ij| < r by brute     */
/* force, in lexicographic order.  Returns the count; writes at most    */
/* cap pairs.  counts (may be NULL) gets the number of neighbours of    */
/* every particle (both ends of each pair).                             */
/* ------------------------------------------------------------------ */
int64_t orc_pairs(const orc_system *s, const double *x, double r, int64_t cap,
                  int32_t *pairs, int32_t *counts)
{
    double r2c = r * r;
    int64_t n = s->n, m = 0;
    if (counts) memset(counts, 0, sizeof(int32_t) * (size_t)n);
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i + 1; j < n; ++j) {
            double d[3];
            double r2 = min_image(&x[3 * i], &x[3 * j], s->box, d);
            if (r2 < r2c) {
                if (m < cap && pairs) { pairs[2 * m] = (int32_t)i; pairs[2 * m + 1] = (int32_t)j; }
                if (counts) { counts[i]++; counts[j]++; }
                ++m;
            }
        }
    return m;
}

/* Neighbours of chosen particles (the rows of the Verlet pair set of       */
/* Sec. 2.1.2 for those particles): for sample q, every j != idx[q] with   */
/* |d_ij| < r, in increasing j, and its r^2 (the same FP64 formula as       */
/* orc_pairs).  Brute force over all j, one sample per thread.  counts[q]   */
/* gets the number of neighbours; at most cap of them are written to        */
/* nbr[q * cap ...] and r2[q * cap ...] (either may be NULL).  Returns the  */
/* largest count.                                                           */
int64_t orc_neighbours_sample(const orc_system *s, const double *x, double r, int64_t n_sample,
                              const int64_t *idx, int64_t cap, int32_t *nbr, double *r2out,
                              int32_t *counts)
{
    const double r2c = r * r;
    for (int64_t q = 0; q < n_sample; ++q)
        if (idx[q] < 0 || idx[q] >= s->n) return -1;
    int64_t mx = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(max : mx)
    for (int64_t q = 0; q < n_sample; ++q) {
        const int64_t i = idx[q];
        int64_t m = 0;
        for (int64_t j = 0; j < s->n; ++j) {
            if (j == i) continue;
            double d[3];
            const double r2 = min_image(&x[3 * i], &x[3 * j], s->box, d);
            if (r2 < r2c) {
                if (m < cap) {
                    if (nbr) nbr[q * cap + m] = (int32_t)j;
                    if (r2out) r2out[q * cap + m] = r2;
                }
                ++m;
            }
        }
        counts[q] = (int32_t)m;
        if (m > mx) mx = m;
    }
    return mx;
}

/* Thread count of the OpenMP loops that follow (0 or less: leave as is). */
void orc_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* Adjoint of velocity Verlet (NVE, pair potential only) for a loss    */
/* L(U_T, K_T, W_T) of the final state, by reverse-mode differentiation */
/* of the map of Fig. 1.  Written from the equations:                  */
/*   pair force on i:  f_ij = g(r) d,  g = 24 eps [2 (s/r)^12 - (s/r)^6] / r^2 */
/*   Jacobian block:   dF_i/dx_j = -(g I + (g'/r) d d^T)  (j != i)     */
/*   parameter terms:  dF_i/d eps = F_i / eps,                          */
/*                     dF_i/d sigma = sum_j (dg/d sigma) d              */
/* with r_cut = rc_over_sigma * sigma moving with sigma (V shifted to  */
/* zero at r_cut, so U and W have no boundary term in sigma); pairs     */
/* that cross r_cut as sigma changes contribute delta terms that a      */
/* pointwise derivative does not see.                                   */
/* ------------------------------------------------------------------ */

/* g(r), g'(r)/r and dg/dsigma for separation r^2 (r < rc). */
static void lj_g_terms(double eps, double sigma, double r2, double *g, double *gpr, double *dgds)
{
    double s2 = sigma * sigma / r2;
    double s6 = s2 * s2 * s2;
    double s12 = s6 * s6;
    *g = 24.0 * eps * (2.0 * s12 - s6) / r2;
    *gpr = 24.0 * eps * (8.0 * s6 - 28.0 * s12) / (r2 * r2);
    *dgds = 24.0 * eps * (24.0 * s12 - 6.0 * s6) / (sigma * r2);
}

/* (J w)_i for the pair forces at x, and the parameter projections
 * pe = sum_i w_i . dF_i/deps and ps = sum_i w_i . dF_i/dsigma. */
void orc_hvp(const orc_system *s, const double *x, const double *w, double *hv, double *pe, double *ps)
{
    int64_t n = s->n;
    double rc2 = s->rc * s->rc;
    double *pe_i = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    double *ps_i = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
        double acc[3] = {0, 0, 0}, F[3] = {0, 0, 0}, Fs[3] = {0, 0, 0};
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double d[3];
            double r2 = min_image(&x[3 * i], &x[3 * j], s->box, d);
            if (!(r2 < rc2)) continue;
            double g, gpr, dgds;
            lj_g_terms(s->eps, s->sigma, r2, &g, &gpr, &dgds);
            double dw[3] = {w[3 * i] - w[3 * j], w[3 * i + 1] - w[3 * j + 1], w[3 * i + 2] - w[3 * j + 2]};
            double ddw = d[0] * dw[0] + d[1] * dw[1] + d[2] * dw[2];
            for (int k = 0; k < 3; ++k) {
                acc[k] += g * dw[k] + gpr * d[k] * ddw;
                F[k] += g * d[k];
                Fs[k] += dgds * d[k];
            }
        }
        for (int k = 0; k < 3; ++k) hv[3 * i + k] = acc[k];
        pe_i[i] = (w[3 * i] * F[0] + w[3 * i + 1] * F[1] + w[3 * i + 2] * F[2]) / s->eps;
        ps_i[i] = w[3 * i] * Fs[0] + w[3 * i + 1] * Fs[1] + w[3 * i + 2] * Fs[2];
    }
    double a = 0, b = 0;
    for (int64_t i = 0; i < n; ++i) { a += pe_i[i]; b += ps_i[i]; }
    free(pe_i);
    free(ps_i);
    *pe = a;
    *ps = b;
}

/* Gradient of L = cU U + cK K + cW W at the final state (x, v):
 *   lx = -cU F + cW dW/dx,  lv = cK m v,
 *   g_eps = (cU U + cW W) / eps,
 *   g_sigma = cU dU/dsigma + cW sum_pairs r^2 dg/dsigma, where dU/dsigma = W / sigma
 *   when r_cut moves with sigma (the shifted energy is a function of r / sigma),
 *   and W / sigma - n_pairs g(r_cut) r_cut^2 / sigma when r_cut is fixed (the
 *   shift V(r_cut) then depends on sigma). */
static int g_rc_fixed = 0;
void orc_set_rc_fixed(int fixed) { g_rc_fixed = fixed; }

void orc_loss_grad(const orc_system *s, const double *x, const double *v, double cU, double cK, double cW,
                   double *lx, double *lv, double *g_eps, double *g_sig)
{
    int64_t n = s->n;
    double rc2 = s->rc * s->rc;
    double U = 0, W = 0, Ws = 0, npair = 0;
    double *Ui = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    double *Pi = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    double *Wi = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    double *Wsi = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
        double F[3] = {0, 0, 0}, dW[3] = {0, 0, 0}, u = 0, wv = 0, ws = 0, np_ = 0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double d[3];
            double r2 = min_image(&x[3 * i], &x[3 * j], s->box, d);
            if (!(r2 < rc2)) continue;
            double g, gpr, dgds;
            lj_g_terms(s->eps, s->sigma, r2, &g, &gpr, &dgds);
            double r = sqrt(r2);
            double vp = orc_lj_energy(r, s->eps, s->sigma);
            if (s->shift) vp -= orc_lj_energy(s->rc, s->eps, s->sigma);
            for (int k = 0; k < 3; ++k) {
                F[k] += g * d[k];
                dW[k] += (2.0 * g + gpr * r2) * d[k];    /* d(g r^2)/dd = (2 g + g' r) d */
            }
            u += 0.5 * vp;
            wv += 0.5 * g * r2;
            ws += 0.5 * r2 * dgds;
            np_ += 0.5;
        }
        for (int k = 0; k < 3; ++k) {
            lx[3 * i + k] = -cU * F[k] + cW * dW[k];
            lv[3 * i + k] = cK * s->mass * v[3 * i + k];
        }
        Ui[i] = u;
        Wi[i] = wv;
        Wsi[i] = ws;
        Pi[i] = np_;
    }
    for (int64_t i = 0; i < n; ++i) { U += Ui[i]; W += Wi[i]; Ws += Wsi[i]; npair += Pi[i]; }
    free(Pi);
    free(Ui);
    free(Wi);
    free(Wsi);
    double dUds = W / s->sigma;
    if (g_rc_fixed && s->shift) {
        double g, gpr, dgds;
        lj_g_terms(s->eps, s->sigma, s->rc * s->rc, &g, &gpr, &dgds);
        dUds -= npair * g * s->rc * s->rc / s->sigma;
    }
    *g_eps = (cU * U + cW * W) / s->eps;
    *g_sig = cU * dUds + cW * Ws;
}

/* Reverse pass through nsteps NVE velocity-Verlet steps from (x0, v0):
 * runs the forward (keeping every position), then the adjoint of each step
 * (half kick, drift, half kick, in reverse).  The loss is
 * L = cU U + cK K + cW W + gx . x_T + gv . v_T at the final state; gx and gv
 * ((N, 3) each, either may be NULL) are the loss's own gradients in the final
 * positions and velocities.  Outputs the final (U, K, W), dL/deps, dL/dsigma,
 * and the adjoints lx0, lv0 of the initial state. */
int orc_vv_adjoint(const orc_system *s, const double *x0, const double *v0, int64_t nsteps,
                   double cU, double cK, double cW, const double *gx, const double *gv, double *euw,
                   double *g_eps, double *g_sig, double *lx0, double *lv0)
{
    int64_t n = s->n;
    size_t sz = (size_t)(3 * n);
    double *X = (double *)malloc(sizeof(double) * sz * (size_t)(nsteps + 1));
    double *v = (double *)malloc(sizeof(double) * sz);
    double *F = (double *)malloc(sizeof(double) * sz);
    double *w = (double *)malloc(sizeof(double) * sz);
    double *hv = (double *)malloc(sizeof(double) * sz);
    if (!X || !v || !F || !w || !hv) { free(X); free(v); free(F); free(w); free(hv); return ORC_ERR_ARG; }
    memcpy(X, x0, sizeof(double) * sz);
    memcpy(v, v0, sizeof(double) * sz);
    double h = 0.5 * s->dt / s->mass;
    orc_forces(s, X, NULL, F, NULL);
    for (int64_t t = 0; t < nsteps; ++t) {
        double *xa = X + sz * (size_t)t, *xb = X + sz * (size_t)(t + 1);
        for (size_t q = 0; q < sz; ++q) {
            v[q] += h * F[q];
            xb[q] = wrap(xa[q] + s->dt * v[q], s->box[q % 3]);
        }
        orc_forces(s, xb, NULL, F, NULL);
        for (size_t q = 0; q < sz; ++q) v[q] += h * F[q];
    }
    double *xT = X + sz * (size_t)nsteps;
    orc_forces(s, xT, v, F, euw);
    double ge, gs;
    double *lx = lx0, *lv = lv0;
    orc_loss_grad(s, xT, v, cU, cK, cW, lx, lv, &ge, &gs);
    for (size_t q = 0; q < sz; ++q) {
        if (gx) lx[q] += gx[q];
        if (gv) lv[q] += gv[q];
    }
    for (int64_t t = nsteps; t >= 0 && nsteps > 0; --t) {
        /* kick(s) at x_t: the first half kick of step t and the second of step t-1 */
        double c = (t == nsteps || t == 0) ? h : 2.0 * h;
        double pe, ps;
        orc_hvp(s, X + sz * (size_t)t, lv, hv, &pe, &ps);
        for (size_t q = 0; q < sz; ++q) lx[q] += c * hv[q];
        ge += c * pe;
        gs += c * ps;
        if (t > 0)   /* drift of step t-1: x_t = x_{t-1} + dt v_half */
            for (size_t q = 0; q < sz; ++q) lv[q] += s->dt * lx[q];
    }
    *g_eps = ge;
    *g_sig = gs;
    free(X); free(v); free(F); free(w); free(hv);
    return ORC_OK;
}
