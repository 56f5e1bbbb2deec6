/*
 * pp_oracle.c -- plain, slow, FP64 CPU oracle for the electrostatic
 * particle-particle (PP) model of electron-bunch expansion in vacuum
 * (Zhang, Ma, Liu, Zhao, "Comparison between electrostatic PP and PIC
 * simulations on electron bunch expansion", arXiv 2502.10640, Sec. 2.1).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check of the
 * package entry file and the CPU-baseline leg of the benchmark may load or
 * call this code.  The GPU product path never does, and this file shares no
 * code, header, constant table or helper with it.
 *
 * Everything is written as the definitions read, with no blocking, fusion or
 * reordering:
 *   - Coulomb pair force, Eq. A, with r_ij = r_i - r_j (repulsive for like
 *     charges; the paper's words "pointing from i to j" contradict its own
 *     formula, and the formula is taken);
 *   - field at particle i from all j != i, Eq. B, specialised to electrons
 *     (Q = q_e w, q_e = -e), Eq. E;
 *   - acceleration a_i = (q_e / m_e) E_i, Eq. D/F (the weight cancels);
 *   - Velocity Verlet, Eq. G then Eq. H;
 *   - emittance, Eq. I, with raw (uncentred) averages over all particles;
 *   - the moment and extreme diagnostics of Figs. 5-6 (x_rms, x_max,
 *     vx_rms, vx_max).
 * Optional Plummer softening eps enters as |r|^2 -> |r|^2 + eps^2 in the
 * field and in the potential (eps = 0 gives Eq. A exactly).  A pair whose
 * softened squared distance is exactly zero contributes nothing (the paper
 * excludes only j == i; coincident distinct particles are read the same way).
 * Particles carry individual weights w_j; the paper uses one common weight.
 *
 * Summation: ascending j with plain "+=", FP64, OpenMP over i only.
 * Compile with -O2 -ffp-contract=off so that no fused multiply-add changes
 * the rounding of the written expressions.
 *
 * Parity pins (closed forms, invariants, published constants) live in the
 * CPU test suite.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>
#include <stdlib.h>

/* CODATA 2018 values; the paper does not print its constants. */
static const double OR_E = 1.602176634e-19;     /* elementary charge, C (exact) */
static const double OR_ME = 9.1093837015e-31;   /* electron mass, kg */
static const double OR_EPS0 = 8.8541878128e-12; /* vacuum permittivity, F/m */
static const double OR_PI = 3.14159265358979323846;

double oracle_const_e(void) { return OR_E; }
double oracle_const_me(void) { return OR_ME; }
double oracle_const_eps0(void) { return OR_EPS0; }
/* Coulomb constant 1/(4 pi eps0), Eq. A. */
double oracle_const_k(void) { return 1.0 / (4.0 * OR_PI * OR_EPS0); }

/*
 * Eq. B / Eq. E: E_i = 1/(4 pi eps0) * sum_{j != i} Q_j (r_i - r_j) / s_ij^{3/2},
 * s_ij = |r_i - r_j|^2 + eps^2, Q_j = q_e w_j, q_e = -e.
 * pos: [N][3] metres; w: [N] weights; E: [N][3] V/m (written).
 * Only the M target indices idx[0..M-1] are computed (E row m belongs to
 * particle idx[m]); idx == NULL means all N particles in order.
 */
void oracle_fields_subset(int64_t N, const double *pos, const double *w,
                          double eps, int64_t M, const int64_t *idx, double *E)
{
    const double k = oracle_const_k();
    const double qe = -OR_E;
    const double eps2 = eps * eps;
    int64_t m;
#pragma omp parallel for schedule(static)
    for (m = 0; m < M; ++m) {
        const int64_t i = idx ? idx[m] : m;
        double ex = 0.0, ey = 0.0, ez = 0.0;
        for (int64_t j = 0; j < N; ++j) {
            if (j == i) continue;
            double dx = pos[3 * i + 0] - pos[3 * j + 0];
            double dy = pos[3 * i + 1] - pos[3 * j + 1];
            double dz = pos[3 * i + 2] - pos[3 * j + 2];
            double s = dx * dx + dy * dy + dz * dz + eps2;
            if (s == 0.0) continue;
            double inv3 = 1.0 / (s * sqrt(s));
            double Qj = qe * w[j];
            ex += Qj * dx * inv3;
            ey += Qj * dy * inv3;
            ez += Qj * dz * inv3;
        }
        E[3 * m + 0] = k * ex;
        E[3 * m + 1] = k * ey;
        E[3 * m + 2] = k * ez;
    }
}

void oracle_fields(int64_t N, const double *pos, const double *w, double eps, double *E)
{
    oracle_fields_subset(N, pos, w, eps, N, NULL, E);
}

/* Eq. D/F: a_i = (q_e / m_e) E_i.  acc: [N][3] m/s^2 (written). */
void oracle_accel(int64_t N, const double *pos, const double *w, double eps, double *acc)
{
    const double qm = -OR_E / OR_ME;
    oracle_fields(N, pos, w, eps, acc);
    for (int64_t i = 0; i < 3 * N; ++i) acc[i] = qm * acc[i];
}

/*
 * Velocity Verlet, Eq. G and Eq. H, nsteps steps of dt.
 * On entry acc must hold a(r) for the entering positions (call oracle_accel
 * first); on return pos, vel, acc hold r, v, a at t + nsteps*dt.
 *   r(t+dt) = r + v dt + a dt^2/2           (Eq. G)
 *   a(t+dt) = (q_e/m_e) E(r(t+dt))           (Eq. F)
 *   v(t+dt) = v + [a(t) + a(t+dt)] dt/2      (Eq. H)
 * scratch: [N][3] doubles supplied by the caller.
 */
void oracle_vv_run(int64_t N, double *pos, double *vel, double *acc,
                   const double *w, double eps, double dt, int64_t nsteps,
                   double *scratch)
{
    const double half_dt2 = dt * dt / 2.0;
    const double half_dt = dt / 2.0;
    for (int64_t n = 0; n < nsteps; ++n) {
        for (int64_t i = 0; i < 3 * N; ++i)
            pos[i] = pos[i] + vel[i] * dt + acc[i] * half_dt2;
        oracle_accel(N, pos, w, eps, scratch);
        for (int64_t i = 0; i < 3 * N; ++i) {
            vel[i] = vel[i] + (acc[i] + scratch[i]) * half_dt;
            acc[i] = scratch[i];
        }
    }
}

/*
 * Electrostatic potential energy, pairs counted once:
 *   PE = 1/2 sum_i sum_{j != i} Q_i Q_j / (4 pi eps0 sqrt(s_ij)).
 */
double oracle_potential_energy(int64_t N, const double *pos, const double *w, double eps)
{
    const double k = oracle_const_k();
    const double eps2 = eps * eps;
    double total = 0.0;
    double *row = (double *)malloc((size_t)(N > 0 ? N : 1) * sizeof(double));
    int64_t i;
#pragma omp parallel for schedule(static)
    for (i = 0; i < N; ++i) {
        double acc = 0.0;
        for (int64_t j = 0; j < N; ++j) {
            if (j == i) continue;
            double dx = pos[3 * i + 0] - pos[3 * j + 0];
            double dy = pos[3 * i + 1] - pos[3 * j + 1];
            double dz = pos[3 * i + 2] - pos[3 * j + 2];
            double s = dx * dx + dy * dy + dz * dz + eps2;
            if (s == 0.0) continue;
            acc += w[j] / sqrt(s);
        }
        row[i] = w[i] * acc;
    }
    for (i = 0; i < N; ++i) total += row[i];
    free(row);
    return 0.5 * k * OR_E * OR_E * total;
}

/*
 * Diagnostics over all particles (out[], in this order):
 *  0 rms_radius  sqrt(<|r - <r>|^2>)           (3D, centred)
 *  1 ke          sum_i 1/2 m_e w_i |v_i|^2
 *  2 px, 3 py, 4 pz   sum_i m_e w_i v_i         (total momentum)
 *  5 emit_x      sqrt(<x^2><vx^2> - <x vx>^2)  (Eq. I, raw averages)
 *  6 x_rms       sqrt(<x^2>)                    (Fig. 5 top)
 *  7 x_max       max_i x_i                      (Fig. 5 bottom)
 *  8 vx_rms      sqrt(<vx^2>)                   (Fig. 6 top)
 *  9 vx_max      max_i vx_i                     (Fig. 6 bottom)
 * 10 cx, 11 cy, 12 cz   centroid <r>
 * Averages <.> are plain means over the N macro-particles, as Eq. I states.
 * Sums run in ascending i.
 */
void oracle_diagnostics(int64_t N, const double *pos, const double *vel,
                        const double *w, double *out)
{
    double cx = 0, cy = 0, cz = 0;
    for (int64_t i = 0; i < N; ++i) {
        cx += pos[3 * i + 0];
        cy += pos[3 * i + 1];
        cz += pos[3 * i + 2];
    }
    cx /= (double)N; cy /= (double)N; cz /= (double)N;
    double r2 = 0, ke = 0, px = 0, py = 0, pz = 0;
    double x2 = 0, vx2 = 0, xvx = 0;
    double xmax = -INFINITY, vxmax = -INFINITY;
    for (int64_t i = 0; i < N; ++i) {
        double dx = pos[3 * i + 0] - cx;
        double dy = pos[3 * i + 1] - cy;
        double dz = pos[3 * i + 2] - cz;
        r2 += dx * dx + dy * dy + dz * dz;
        double vx = vel[3 * i + 0], vy = vel[3 * i + 1], vz = vel[3 * i + 2];
        double m = OR_ME * w[i];
        ke += 0.5 * m * (vx * vx + vy * vy + vz * vz);
        px += m * vx;
        py += m * vy;
        pz += m * vz;
        double x = pos[3 * i + 0];
        x2 += x * x;
        vx2 += vx * vx;
        xvx += x * vx;
        if (x > xmax) xmax = x;
        if (vx > vxmax) vxmax = vx;
    }
    double n = (double)N;
    double mx2 = x2 / n, mvx2 = vx2 / n, mxvx = xvx / n;
    double e2 = mx2 * mvx2 - mxvx * mxvx;
    out[0] = sqrt(r2 / n);
    out[1] = ke;
    out[2] = px; out[3] = py; out[4] = pz;
    out[5] = sqrt(e2 > 0.0 ? e2 : 0.0);
    out[6] = sqrt(mx2);
    out[7] = xmax;
    out[8] = sqrt(mvx2);
    out[9] = vxmax;
    out[10] = cx; out[11] = cy; out[12] = cz;
}
