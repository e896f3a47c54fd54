/*
 * FP64 CPU oracle for the improved multiple-relaxation-time (MRT) pseudopotential
 * lattice Boltzmann step of Li, Luo & Li, "Lattice Boltzmann modeling of multiphase
 * flows at large density ratio with an improved pseudopotential model"
 * (arXiv:1211.6932).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the CUDA
 * library is checked against.  Nothing in the product path may link, load or call it;
 * only the test-suite, the smoke check and the CPU-baseline leg of the benchmark do.
 * It shares no code, table or header with the CUDA path.
 *
 * Every node update follows the paper's order, in double precision:
 *   1. density              rho = sum_a f_a                           (Sec. II, Eq. 6)
 *   2. pseudopotential      psi = sqrt(2 (p_EOS - rho c_s^2) / (G c^2))  (Eq. 24)
 *      with the Carnahan-Starling equation of state                      (Eq. 30)
 *   3. interaction force    F = -G psi(x) sum_a w(|e_a|^2) psi(x+e_a) e_a (Eq. 7)
 *   4. velocity             rho v = sum_a e_a f_a + F/2                (Eq. 6)
 *   5. moments              m = M f,  m_eq from Eq. 3
 *   6. forcing in moment space, improved scheme                        (Eq. 25)
 *   7. collision            m* = m - Lambda (m - m_eq) + (I - Lambda/2) S   (Eq. 4)
 *   8. back to velocities   f* = M^{-1} m*                              (after Eq. 5)
 *   9. streaming            f_a(x + e_a, t+1) = f*_a(x, t)              (Eq. 5)
 *
 * Readings of points the paper leaves open (each one is listed in the design notes):
 *   - M is not printed in the paper; it is the orthogonal D2Q9 matrix whose rows are
 *     ordered (rho, e, eps, j_x, q_x, j_y, q_y, p_xx, p_xy) so that M f_eq equals the
 *     moment equilibria of Eq. 3.  M^{-1} = M^T diag(1/|row|^2).
 *   - Eq. 2 lists inverse relaxation times; the nine rates s[0..8] are those inverses.
 *     The tau_e and tau_varsigma of Eq. 25 are 1/s[1] and 1/s[2].
 *   - |F|^2 / psi^2 in Eq. 25 is evaluated as |F/psi|^2, where F/psi is the sum of
 *     Eq. 7 without the leading psi(x); this is the same number for psi != 0 and avoids
 *     0/0 where psi vanishes.
 *   - A negative argument under the square root of Eq. 24 is clamped to zero.
 *   - Viscosity modes (Sec. IV C): constant (s[7], s[8] as given); step (nu_l where
 *     rho >= rho_c, nu_v below); linear (relaxation time linear in rho between rho_v
 *     and rho_l, clamped).  In the last two s[7] = s[8] = 1/(3 nu + 1/2) (Eq. 10 with
 *     c_s^2 = 1/3, delta_t = 1).
 *   - Walls (Sec. IV C, no-slip in y): halfway bounce-back at y = -1/2 and
 *     y = ny - 1/2; psi at a ghost row equals psi of the adjacent fluid row.
 *
 * Lattice units throughout: c = delta_t = 1, c_s^2 = 1/3.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define Q 9

/* D2Q9 velocities, in the order used by the moment basis of Eq. 3. */
static const int EX[Q] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[Q] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const int OPP[Q] = {0, 3, 4, 1, 2, 7, 8, 5, 6};

/* Interaction weights of Eq. 7 for nearest neighbours: w(1) = 1/3, w(2) = 1/12. */
static double force_weight(int a) {
    int e2 = EX[a] * EX[a] + EY[a] * EY[a];
    if (e2 == 1) return 1.0 / 3.0;
    if (e2 == 2) return 1.0 / 12.0;
    return 0.0;
}

/* Transformation matrix M (rows: rho, e, eps, j_x, q_x, j_y, q_y, p_xx, p_xy). */
static const double M[Q][Q] = {
    { 1,  1,  1,  1,  1,  1,  1,  1,  1},
    {-4, -1, -1, -1, -1,  2,  2,  2,  2},
    { 4, -2, -2, -2, -2,  1,  1,  1,  1},
    { 0,  1,  0, -1,  0,  1, -1, -1,  1},
    { 0, -2,  0,  2,  0,  1, -1, -1,  1},
    { 0,  0,  1,  0, -1,  1,  1, -1, -1},
    { 0,  0, -2,  0,  2,  1,  1, -1, -1},
    { 0,  1, -1,  1, -1,  0,  0,  0,  0},
    { 0,  0,  0,  0,  0,  1, -1,  1, -1},
};

typedef struct {
    int nx, ny;
    double a, b, R, T;     /* Carnahan-Starling EOS, Eq. 30 */
    double G;              /* interaction strength, Eq. 7 */
    double sigma;          /* improved-forcing parameter, Eq. 25 */
    double s[Q];           /* relaxation rates (inverse times), Eq. 2 */
    int visc_mode;         /* 0 constant, 1 step at rho_c, 2 linear in rho */
    double nu_l, nu_v;     /* liquid / vapour kinematic viscosity */
    double rho_c;          /* switch density of the step mode */
    double rho_l, rho_v;   /* end points of the linear mode */
    int walls;             /* 0 periodic in y, 1 bounce-back walls in y */
} oracle_params;

/* M^{-1} = M^T diag(1 / sum_b M[i][b]^2), valid because M is orthogonal. */
static void minv_build(double Minv[Q][Q]) {
    for (int i = 0; i < Q; ++i) {
        double n2 = 0.0;
        for (int b = 0; b < Q; ++b) n2 += M[i][b] * M[i][b];
        for (int b = 0; b < Q; ++b) Minv[b][i] = M[i][b] / n2;
    }
}

/* Carnahan-Starling pressure, Eq. 30. */
double oracle_p_eos(double rho, double a, double b, double R, double T) {
    double x = b * rho / 4.0;
    double num = 1.0 + x + x * x - x * x * x;
    double den = (1.0 - x) * (1.0 - x) * (1.0 - x);
    return rho * R * T * num / den - a * rho * rho;
}

/* Pseudopotential from the EOS, Eq. 24 (c = 1, c_s^2 = 1/3). */
double oracle_psi(double rho, double a, double b, double R, double T, double G) {
    double arg = 2.0 * (oracle_p_eos(rho, a, b, R, T) - rho / 3.0) / G;
    if (arg < 0.0) arg = 0.0;
    return sqrt(arg);
}

/* Stress-moment relaxation rate for the chosen viscosity mode (Eq. 10, Sec. IV C). */
static double stress_rate(const oracle_params* p, double rho, int which) {
    if (p->visc_mode == 0) return p->s[which];
    if (p->visc_mode == 1) {
        double nu = (rho >= p->rho_c) ? p->nu_l : p->nu_v;
        return 1.0 / (3.0 * nu + 0.5);
    }
    double tau_l = 3.0 * p->nu_l + 0.5, tau_v = 3.0 * p->nu_v + 0.5;
    double frac = (rho - p->rho_v) / (p->rho_l - p->rho_v);
    if (frac < 0.0) frac = 0.0;
    if (frac > 1.0) frac = 1.0;
    return 1.0 / (tau_v + frac * (tau_l - tau_v));
}

static int wrap(int i, int n) {
    i %= n;
    return i < 0 ? i + n : i;
}

/* psi at lattice position (x, y), y possibly a ghost row next to a wall. */
static double psi_at(const oracle_params* p, const double* psi, int x, int y) {
    x = wrap(x, p->nx);
    if (p->walls) {
        if (y < 0) y = 0;
        if (y >= p->ny) y = p->ny - 1;
    } else {
        y = wrap(y, p->ny);
    }
    return psi[(size_t)y * p->nx + x];
}

/*
 * Per-node quantities of Eqs. 6 and 7 at the current time: rho, psi, F/psi and v.
 * Arrays are (ny, nx), row-major.  f is (Q, ny, nx).
 */
static void macroscopic(const oracle_params* p, const double* f, double* rho, double* psi,
                        double* fpx, double* fpy, double* ux, double* uy) {
    const int nx = p->nx, ny = p->ny;
    const size_t N = (size_t)nx * ny;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            size_t n = (size_t)y * nx + x;
            double r = 0.0;
            for (int a = 0; a < Q; ++a) r += f[a * N + n];
            rho[n] = r;
            psi[n] = oracle_psi(r, p->a, p->b, p->R, p->T, p->G);
        }
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            size_t n = (size_t)y * nx + x;
            double sx = 0.0, sy = 0.0;
            for (int a = 1; a < Q; ++a) {
                double w = force_weight(a) * psi_at(p, psi, x + EX[a], y + EY[a]);
                sx += w * EX[a];
                sy += w * EY[a];
            }
            fpx[n] = -p->G * sx; /* F / psi(x) */
            fpy[n] = -p->G * sy;
            double jx = 0.0, jy = 0.0;
            for (int a = 0; a < Q; ++a) {
                jx += EX[a] * f[a * N + n];
                jy += EY[a] * f[a * N + n];
            }
            double Fx = psi[n] * fpx[n], Fy = psi[n] * fpy[n];
            ux[n] = (jx + 0.5 * Fx) / rho[n];
            uy[n] = (jy + 0.5 * Fy) / rho[n];
        }
}

/* Moment equilibria, Eq. 3. */
static void moment_eq(double rho, double vx, double vy, double meq[Q]) {
    double v2 = vx * vx + vy * vy;
    meq[0] = rho;
    meq[1] = rho * (-2.0 + 3.0 * v2);
    meq[2] = rho * (1.0 - 3.0 * v2);
    meq[3] = rho * vx;
    meq[4] = -rho * vx;
    meq[5] = rho * vy;
    meq[6] = -rho * vy;
    meq[7] = rho * (vx * vx - vy * vy);
    meq[8] = rho * vx * vy;
}

/* Forcing term in moment space, improved scheme of Eq. 25 (Eq. 9 when sigma = 0). */
static void forcing(const oracle_params* p, double vx, double vy, double Fx, double Fy,
                    double F2_over_psi2, double S[Q]) {
    double vF = vx * Fx + vy * Fy;
    double tau_e = 1.0 / p->s[1], tau_z = 1.0 / p->s[2];
    S[0] = 0.0;
    S[1] = 6.0 * vF + 12.0 * p->sigma * F2_over_psi2 / (tau_e - 0.5);
    S[2] = -6.0 * vF - 12.0 * p->sigma * F2_over_psi2 / (tau_z - 0.5);
    S[3] = Fx;
    S[4] = -Fx;
    S[5] = Fy;
    S[6] = -Fy;
    S[7] = 2.0 * (vx * Fx - vy * Fy);
    S[8] = vx * Fy + vy * Fx;
}

/* One time step.  f (Q, ny, nx) -> fnew; both are at the same stage (pre-collision). */
static void one_step(const oracle_params* p, const double* f, double* fnew, double* rho,
                     double* psi, double* fpx, double* fpy, double* ux, double* uy,
                     double* fstar) {
    const int nx = p->nx, ny = p->ny;
    const size_t N = (size_t)nx * ny;
    double Minv[Q][Q];
    minv_build(Minv);
    macroscopic(p, f, rho, psi, fpx, fpy, ux, uy);
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            size_t n = (size_t)y * nx + x;
            double fl[Q], m[Q], meq[Q], S[Q], ms[Q], lam[Q];
            for (int a = 0; a < Q; ++a) fl[a] = f[a * N + n];
            for (int i = 0; i < Q; ++i) {
                double acc = 0.0;
                for (int a = 0; a < Q; ++a) acc += M[i][a] * fl[a];
                m[i] = acc;
            }
            moment_eq(rho[n], ux[n], uy[n], meq);
            double Fx = psi[n] * fpx[n], Fy = psi[n] * fpy[n];
            forcing(p, ux[n], uy[n], Fx, Fy, fpx[n] * fpx[n] + fpy[n] * fpy[n], S);
            for (int i = 0; i < Q; ++i) lam[i] = p->s[i];
            lam[7] = stress_rate(p, rho[n], 7);
            lam[8] = stress_rate(p, rho[n], 8);
            for (int i = 0; i < Q; ++i)
                ms[i] = m[i] - lam[i] * (m[i] - meq[i]) + (1.0 - 0.5 * lam[i]) * S[i];
            for (int a = 0; a < Q; ++a) {
                double acc = 0.0;
                for (int i = 0; i < Q; ++i) acc += Minv[a][i] * ms[i];
                fstar[a * N + n] = acc;
            }
        }
    /* Streaming, Eq. 5: f_a(x + e_a) <- f*_a(x); halfway bounce-back at walls. */
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            size_t n = (size_t)y * nx + x;
            for (int a = 0; a < Q; ++a) {
                int xd = wrap(x + EX[a], nx);
                int yd = y + EY[a];
                if (p->walls && (yd < 0 || yd >= ny)) {
                    fnew[OPP[a] * N + n] = fstar[a * N + n];
                } else {
                    yd = wrap(yd, ny);
                    fnew[a * N + (size_t)yd * nx + xd] = fstar[a * N + n];
                }
            }
        }
}

static double* alloc_d(size_t n) { return (double*)malloc(n * sizeof(double)); }

/*
 * Advance nsteps time steps.  f_in and f_out are (Q, ny, nx) arrays; they may alias.
 * Returns 0 on success, -1 on bad arguments, -2 on allocation failure.
 */
int oracle_run(const oracle_params* p, const double* f_in, double* f_out, int nsteps) {
    if (!p || p->nx < 1 || p->ny < 1 || nsteps < 0) return -1;
    const size_t N = (size_t)p->nx * p->ny;
    double *a = alloc_d(Q * N), *b = alloc_d(Q * N), *fs = alloc_d(Q * N);
    double *rho = alloc_d(N), *psi = alloc_d(N), *fpx = alloc_d(N), *fpy = alloc_d(N);
    double *ux = alloc_d(N), *uy = alloc_d(N);
    int rc = 0;
    if (!a || !b || !fs || !rho || !psi || !fpx || !fpy || !ux || !uy) {
        rc = -2;
        goto done;
    }
    memcpy(a, f_in, Q * N * sizeof(double));
    for (int s = 0; s < nsteps; ++s) {
        one_step(p, a, b, rho, psi, fpx, fpy, ux, uy, fs);
        double* t = a; a = b; b = t;
    }
    memcpy(f_out, a, Q * N * sizeof(double));
done:
    free(a); free(b); free(fs); free(rho); free(psi); free(fpx); free(fpy); free(ux); free(uy);
    return rc;
}

/*
 * Macroscopic fields of Eq. 6 at the current time, plus psi (Eq. 24) and the force of
 * Eq. 7.  Any output pointer may be NULL.
 */
int oracle_fields(const oracle_params* p, const double* f, double* rho_out, double* ux_out,
                  double* uy_out, double* psi_out, double* Fx_out, double* Fy_out) {
    if (!p || p->nx < 1 || p->ny < 1) return -1;
    const size_t N = (size_t)p->nx * p->ny;
    double *rho = alloc_d(N), *psi = alloc_d(N), *fpx = alloc_d(N), *fpy = alloc_d(N);
    double *ux = alloc_d(N), *uy = alloc_d(N);
    int rc = 0;
    if (!rho || !psi || !fpx || !fpy || !ux || !uy) {
        rc = -2;
        goto done;
    }
    macroscopic(p, f, rho, psi, fpx, fpy, ux, uy);
    for (size_t n = 0; n < N; ++n) {
        if (rho_out) rho_out[n] = rho[n];
        if (ux_out) ux_out[n] = ux[n];
        if (uy_out) uy_out[n] = uy[n];
        if (psi_out) psi_out[n] = psi[n];
        if (Fx_out) Fx_out[n] = psi[n] * fpx[n];
        if (Fy_out) Fy_out[n] = psi[n] * fpy[n];
    }
done:
    free(rho); free(psi); free(fpx); free(fpy); free(ux); free(uy);
    return rc;
}

/*
 * Initial populations f = M^{-1} m_eq(rho, v) (the equilibrium whose moments are Eq. 3),
 * from (ny, nx) fields rho, ux, uy.  f is (Q, ny, nx).
 */
int oracle_equilibrium(int nx, int ny, const double* rho, const double* ux, const double* uy,
                       double* f) {
    if (nx < 1 || ny < 1) return -1;
    const size_t N = (size_t)nx * ny;
    double Minv[Q][Q];
    minv_build(Minv);
    for (size_t n = 0; n < N; ++n) {
        double meq[Q];
        moment_eq(rho[n], ux[n], uy[n], meq);
        for (int a = 0; a < Q; ++a) {
            double acc = 0.0;
            for (int i = 0; i < Q; ++i) acc += Minv[a][i] * meq[i];
            f[a * N + n] = acc;
        }
    }
    return 0;
}

/* Read-only access to the oracle's lattice tables, for the identity tests. */
void oracle_tables(int* ex, int* ey, int* opp, double* w, double* m) {
    for (int a = 0; a < Q; ++a) {
        ex[a] = EX[a];
        ey[a] = EY[a];
        opp[a] = OPP[a];
        w[a] = force_weight(a);
    }
    for (int i = 0; i < Q; ++i)
        for (int a = 0; a < Q; ++a) m[i * Q + a] = M[i][a];
}

/* Number of OpenMP threads the oracle uses (1 when built without OpenMP). */
int oracle_threads(void) {
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
