/*
 * Plain FP64 CPU oracle of the D3Q19 single-relaxation-time pseudo-potential
 * (Shan-Chen) lattice Boltzmann step of Chiappini, Xue, Falcucci, Sbragaglia,
 * "Ligament break-up simulation through pseudo-potential Lattice Boltzmann
 * Method" (arXiv:1904.11792).
 *
 * TEST INFRASTRUCTURE ONLY.  This library exists to check the GPU path.  Only
 * the test-suite, the smoke check and the benchmark's CPU-baseline leg may
 * load it.  It shares no code, header, table or generator with the CUDA
 * library, and it never calls it.
 *
 * Every routine is the plain definition written out: one loop over nodes,
 * one loop over the 19 directions, no blocking or fusion.  The time step
 * follows the paper's order (section "Numerical model"):
 *   Eq. 4  rho = sum_a f_a,  rho*u = sum_a c_a f_a
 *   (text after Eq. 5)  psi = rho0 * (1 - exp(-rho/rho0))
 *   Eq. 5  F = -G psi(x) sum_a w_a psi(x + c_a) c_a
 *   Eq. 6  u' = u + tau F / rho
 *   Eq. 2  f_eq(rho, u')   (with the leading "1 +", see reading R1 below)
 *   Eq. 3  f_a(x + c_a, t + 1) = f_a - (f_a - f_eq_a) / tau
 *
 * Readings of the paper taken here (each also listed in the design notes):
 *   R1  Eq. 2 as printed has no zeroth-order term; the standard second-order
 *       equilibrium w rho [1 + c.u/cs2 + (c.u)^2/(2 cs2^2) - u.u/(2 cs2)] is
 *       used so that sum_a f_eq = rho, as Eq. 4 requires.
 *   R2  The force enters only through the velocity shift of Eq. 6; the extra
 *       F_a term of Eq. 3 is taken as zero (no double forcing).
 *   R3  u in Eq. 6 is the bare u = j / rho of Eq. 4.
 *   R4  G is signed; attraction (phase separation) needs G < 0.  The paper's
 *       "G0 = 5.3" is G = -5.3.
 *   R5  The weights of Eq. 5 are the lattice weights w_a.
 *   R6  D3Q19 weights 1/3, 1/18, 1/36 and cs^2 = 1/3 ("normalised to unity").
 *   R7  Exported velocity is u = (j + F/2) / rho.
 *   R8  psi at all neighbours comes from the same pre-collision state.
 *   R11 Ligament profile rho_v + (rho_l - rho_v)/2 [1 - tanh(2 (r - R(x))/W)].
 *   R12 Cylinder axis at y = (ny-1)/2, z = (nz-1)/2.
 *   R13 Initial populations f_a = w_a rho (zero velocity).
 *
 * Population layout: f[a * N + i], i = x + nx * (y + ny * z), the values are
 * the pre-collision populations at node i.  Direction order (the library's
 * canonical order): 0 rest; 1..6 = +x,-x,+y,-y,+z,-z; 7..18 the twelve
 * diagonals in opposite pairs (+x+y,-x-y), (+x-y,-x+y), (+x+z,-x-z),
 * (+x-z,-x+z), (+y+z,-y-z), (+y-z,-y+z).
 *
 * Built with -O2 -ffp-contract=off so results are the same on x86-64 and
 * aarch64.  OpenMP (optional) only splits node loops whose iterations write
 * disjoint outputs, so threaded and serial results are identical.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q 19

/* D3Q19 velocity set (reading R6). */
static const int CV[Q][3] = {
    {0, 0, 0},
    {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},  {0, 0, -1},
    {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
    {1, 0, 1},  {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};

static const double WT[Q] = {
    1.0 / 3.0,
    1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0,
    1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0,
    1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

static const int OPPOSITE[Q] = {0, 2, 1, 4, 3, 6, 5, 8, 7, 10, 9,
                                12, 11, 14, 13, 16, 15, 18, 17};

static const double CS2 = 1.0 / 3.0; /* lattice speed of sound squared, R6 */

#define PAR_MIN_NODES 32768

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_num_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* Exports the lattice tables: c[a*3 + k], w[a], opp[a]. */
void orc_lattice(int *c, double *w, int *opp) {
    for (int a = 0; a < Q; ++a) {
        for (int k = 0; k < 3; ++k) c[a * 3 + k] = CV[a][k];
        w[a] = WT[a];
        opp[a] = OPPOSITE[a];
    }
}

/* Periodic wrap of a coordinate; every caller passes a in [-n, 2n). */
static inline int wrap(int a, int n) {
    return a < 0 ? a + n : (a >= n ? a - n : a);
}

static inline size_t node_index(int x, int y, int z, int nx, int ny) {
    return (size_t)x + (size_t)nx * ((size_t)y + (size_t)ny * (size_t)z);
}

/* Pseudo-potential psi(rho) (definition after Eq. 5).  form 0:
 * rho0 (1 - exp(-rho/rho0)); form 1: psi = rho (a test functional). */
double orc_psi(double rho, int form, double rho0) {
    if (form == 1) return rho;
    return rho0 * (1.0 - exp(-rho / rho0));
}

/* Second-order equilibrium, Eq. 2 with the "1 +" of reading R1. */
void orc_feq(double rho, const double *u, double *feq) {
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int a = 0; a < Q; ++a) {
        double cu = CV[a][0] * u[0] + CV[a][1] * u[1] + CV[a][2] * u[2];
        feq[a] = WT[a] * rho *
                 (1.0 + cu / CS2 + (cu * cu) / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
    }
}

/* Eq. 4: zeroth and first moments of the populations at node i. */
static void node_moments(const double *f, size_t N, size_t i, double *rho, double j[3]) {
    double r = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
    for (int a = 0; a < Q; ++a) {
        double fa = f[(size_t)a * N + i];
        r += fa;
        jx += CV[a][0] * fa;
        jy += CV[a][1] * fa;
        jz += CV[a][2] * fa;
    }
    *rho = r;
    j[0] = jx;
    j[1] = jy;
    j[2] = jz;
}

/* psi field of the whole lattice from the pre-collision populations. */
static void psi_field(int nx, int ny, int nz, int psi_form, double rho0, const double *f,
                      double *psi) {
    size_t N = (size_t)nx * ny * nz;
    long long n = (long long)N;
#pragma omp parallel for if (N > PAR_MIN_NODES) schedule(static)
    for (long long ii = 0; ii < n; ++ii) {
        double rho, j[3];
        node_moments(f, N, (size_t)ii, &rho, j);
        psi[ii] = orc_psi(rho, psi_form, rho0);
    }
}

/* Eq. 5: F(x) = -G psi(x) sum_a w_a psi(x + c_a) c_a, periodic lattice. */
static void node_force(int nx, int ny, int nz, const double *psi, int x, int y, int z, double G,
                       double F[3]) {
    double s[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < Q; ++a) {
        size_t nb = node_index(wrap(x + CV[a][0], nx), wrap(y + CV[a][1], ny),
                               wrap(z + CV[a][2], nz), nx, ny);
        for (int k = 0; k < 3; ++k) s[k] += WT[a] * psi[nb] * CV[a][k];
    }
    double p = psi[node_index(x, y, z, nx, ny)];
    for (int k = 0; k < 3; ++k) F[k] = -G * p * s[k];
}

/* Collision at one node (Eqs. 4, 5, 6, 2, 3): post-collision values fstar[a]. */
static void node_collide(int nx, int ny, int nz, double tau, double G, const double *f,
                         const double *psi, int x, int y, int z, double fstar[Q]) {
    size_t N = (size_t)nx * ny * nz;
    size_t i = node_index(x, y, z, nx, ny);
    double rho, j[3], F[3], u[3], feq[Q];
    node_moments(f, N, i, &rho, j);
    node_force(nx, ny, nz, psi, x, y, z, G, F);
    for (int k = 0; k < 3; ++k) u[k] = j[k] / rho + F[k] * tau / rho; /* Eq. 6, R3 */
    orc_feq(rho, u, feq);
    for (int a = 0; a < Q; ++a) {
        double fa = f[(size_t)a * N + i];
        fstar[a] = fa - (fa - feq[a]) / tau; /* Eq. 3, R2 */
    }
}

/*
 * nsteps time steps in place on f (19*N doubles, layout above).  Two
 * separate arrays (A-B): psi for every node first (R8), then collide and
 * stream each node into the second array.  Returns 0, or -1 on allocation
 * failure.
 */
int orc_step(int nx, int ny, int nz, double tau, double G, int psi_form, double rho0, double *f,
             int nsteps) {
    size_t N = (size_t)nx * ny * nz;
    double *psi = (double *)malloc(N * sizeof(double));
    double *g = (double *)malloc((size_t)Q * N * sizeof(double));
    if (!psi || !g) {
        free(psi);
        free(g);
        return -1;
    }
    double *cur = f, *nxt = g;
    for (int s = 0; s < nsteps; ++s) {
        psi_field(nx, ny, nz, psi_form, rho0, cur, psi);
        long long rows = (long long)ny * nz;
#pragma omp parallel for if (N > PAR_MIN_NODES) schedule(static)
        for (long long r = 0; r < rows; ++r) {
            int y = (int)(r % ny), z = (int)(r / ny);
            for (int x = 0; x < nx; ++x) {
                double fstar[Q];
                node_collide(nx, ny, nz, tau, G, cur, psi, x, y, z, fstar);
                for (int a = 0; a < Q; ++a) {
                    size_t d = node_index(wrap(x + CV[a][0], nx), wrap(y + CV[a][1], ny),
                                          wrap(z + CV[a][2], nz), nx, ny);
                    nxt[(size_t)a * N + d] = fstar[a];
                }
            }
        }
        double *t = cur;
        cur = nxt;
        nxt = t;
    }
    if (cur != f) memcpy(f, cur, (size_t)Q * N * sizeof(double));
    free(psi);
    free(g);
    return 0;
}

/*
 * Multiple-relaxation-time collision: the operator the paper names as its
 * next step (section "Conclusions": MRT keeps the density ratio fixed while
 * the viscosity changes).  It is not specified in the paper; this follows the
 * standard D3Q19 MRT of d'Humieres, Ginzburg, Krafczyk, Lallemand and Luo
 * (Phil. Trans. R. Soc. A 360, 2002) with the forcing of Guo, Zheng and Shi
 * (Phys. Rev. E 65, 046308, 2002) written in moment space:
 *   m = M f,  m_eq = M f_eq(rho, u),  s_F = M F_guo,  u = (j + F/2) / rho,
 *   F_guo_a = w_a [ (c_a - u).F / cs2 + (c_a.u)(c_a.F) / cs2^2 ],
 *   m* = m - S (m - m_eq) + (I - S/2) s_F,   f* = M^-1 m*,
 * with F the Shan-Chen force of Eq. 5 and f_eq the equilibrium of Eq. 2
 * (reading R1).  S = diag(rates[0..18]).
 *
 * Rows of M: polynomials of the velocity c (c2 = c.c) evaluated on the 19
 * lattice velocities, in this order:
 *   0 1 (density)   1 19 c2 - 30 (energy)   2 (21 c2^2 - 53 c2 + 24)/2
 *   3 cx   4 (5 c2 - 9) cx   5 cy   6 (5 c2 - 9) cy   7 cz   8 (5 c2 - 9) cz
 *   9 3 cx^2 - c2   10 (3 c2 - 5)(3 cx^2 - c2)   11 cy^2 - cz^2
 *   12 (3 c2 - 5)(cy^2 - cz^2)   13 cx cy   14 cy cz   15 cx cz
 *   16 (cy^2 - cz^2) cx   17 (cz^2 - cx^2) cy   18 (cx^2 - cy^2) cz
 * The rows are mutually orthogonal, so M^-1 = M^T diag(1 / |row|^2).
 */
static double mrt_row(int k, const int c[3]) {
    double x = c[0], y = c[1], z = c[2], c2 = x * x + y * y + z * z;
    switch (k) {
        case 0: return 1.0;
        case 1: return 19.0 * c2 - 30.0;
        case 2: return (21.0 * c2 * c2 - 53.0 * c2 + 24.0) / 2.0;
        case 3: return x;
        case 4: return (5.0 * c2 - 9.0) * x;
        case 5: return y;
        case 6: return (5.0 * c2 - 9.0) * y;
        case 7: return z;
        case 8: return (5.0 * c2 - 9.0) * z;
        case 9: return 3.0 * x * x - c2;
        case 10: return (3.0 * c2 - 5.0) * (3.0 * x * x - c2);
        case 11: return y * y - z * z;
        case 12: return (3.0 * c2 - 5.0) * (y * y - z * z);
        case 13: return x * y;
        case 14: return y * z;
        case 15: return x * z;
        case 16: return (y * y - z * z) * x;
        case 17: return (z * z - x * x) * y;
        default: return (x * x - y * y) * z;
    }
}

/* M (19 x 19, row-major, M[k*19 + a] = row k at velocity a). */
void orc_mrt_matrix(double *M) {
    for (int k = 0; k < Q; ++k)
        for (int a = 0; a < Q; ++a) M[k * Q + a] = mrt_row(k, CV[a]);
}

/* Guo forcing populations F_guo_a for velocity u and force F. */
static void guo_source(const double u[3], const double F[3], double src[Q]) {
    for (int a = 0; a < Q; ++a) {
        double cu = CV[a][0] * u[0] + CV[a][1] * u[1] + CV[a][2] * u[2];
        double cF = CV[a][0] * F[0] + CV[a][1] * F[1] + CV[a][2] * F[2];
        double uF = u[0] * F[0] + u[1] * F[1] + u[2] * F[2];
        src[a] = WT[a] * ((cF - uF) / CS2 + cu * cF / (CS2 * CS2));
    }
}

/* Collision of one node with the MRT operator above (rates = diag S). */
static void node_collide_mrt(int nx, int ny, int nz, const double *rates, double G,
                             const double *M, const double *Minv, const double *f,
                             const double *psi, int x, int y, int z, double fstar[Q]) {
    size_t N = (size_t)nx * ny * nz;
    size_t i = node_index(x, y, z, nx, ny);
    double rho, j[3], F[3], u[3], feq[Q], src[Q], fl[Q];
    node_moments(f, N, i, &rho, j);
    node_force(nx, ny, nz, psi, x, y, z, G, F);
    for (int k = 0; k < 3; ++k) u[k] = (j[k] + 0.5 * F[k]) / rho;
    orc_feq(rho, u, feq);
    guo_source(u, F, src);
    for (int a = 0; a < Q; ++a) fl[a] = f[(size_t)a * N + i];
    double mstar[Q];
    for (int k = 0; k < Q; ++k) {
        double m = 0.0, meq = 0.0, sF = 0.0;
        for (int a = 0; a < Q; ++a) {
            m += M[k * Q + a] * fl[a];
            meq += M[k * Q + a] * feq[a];
            sF += M[k * Q + a] * src[a];
        }
        mstar[k] = m - rates[k] * (m - meq) + (1.0 - 0.5 * rates[k]) * sF;
    }
    for (int a = 0; a < Q; ++a) {
        double v = 0.0;
        for (int k = 0; k < Q; ++k) v += Minv[a * Q + k] * mstar[k];
        fstar[a] = v;
    }
}

/* SRT collision with the same Guo forcing, written in velocity space:
 * f* = f - (f - f_eq(rho, u)) / tau + (1 - 1/(2 tau)) F_guo, u = (j + F/2)/rho. */
static void node_collide_bgk_guo(int nx, int ny, int nz, double tau, double G, const double *f,
                                 const double *psi, int x, int y, int z, double fstar[Q]) {
    size_t N = (size_t)nx * ny * nz;
    size_t i = node_index(x, y, z, nx, ny);
    double rho, j[3], F[3], u[3], feq[Q], src[Q];
    node_moments(f, N, i, &rho, j);
    node_force(nx, ny, nz, psi, x, y, z, G, F);
    for (int k = 0; k < 3; ++k) u[k] = (j[k] + 0.5 * F[k]) / rho;
    orc_feq(rho, u, feq);
    guo_source(u, F, src);
    for (int a = 0; a < Q; ++a) {
        double fa = f[(size_t)a * N + i];
        fstar[a] = fa - (fa - feq[a]) / tau + (1.0 - 0.5 / tau) * src[a];
    }
}

/*
 * nsteps A-B steps with the MRT collision (rates: the 19 diagonal entries
 * of S) or, when rates is NULL, with the velocity-space SRT-Guo collision of
 * relaxation time tau.  Same psi pass and streaming as orc_step.
 */
int orc_step_forcing(int nx, int ny, int nz, double tau, const double *rates, double G, int psi_form,
                     double rho0, double *f, int nsteps) {
    size_t N = (size_t)nx * ny * nz;
    double *psi = (double *)malloc(N * sizeof(double));
    double *g = (double *)malloc((size_t)Q * N * sizeof(double));
    double M[Q * Q], Minv[Q * Q];
    if (!psi || !g) {
        free(psi);
        free(g);
        return -1;
    }
    orc_mrt_matrix(M);
    for (int k = 0; k < Q; ++k) {
        double n2 = 0.0;
        for (int a = 0; a < Q; ++a) n2 += M[k * Q + a] * M[k * Q + a];
        for (int a = 0; a < Q; ++a) Minv[a * Q + k] = M[k * Q + a] / n2;
    }
    double *cur = f, *nxt = g;
    for (int s = 0; s < nsteps; ++s) {
        psi_field(nx, ny, nz, psi_form, rho0, cur, psi);
        long long rows = (long long)ny * nz;
#pragma omp parallel for if (N > PAR_MIN_NODES) schedule(static)
        for (long long r = 0; r < rows; ++r) {
            int y = (int)(r % ny), z = (int)(r / ny);
            for (int x = 0; x < nx; ++x) {
                double fstar[Q];
                if (rates)
                    node_collide_mrt(nx, ny, nz, rates, G, M, Minv, cur, psi, x, y, z, fstar);
                else
                    node_collide_bgk_guo(nx, ny, nz, tau, G, cur, psi, x, y, z, fstar);
                for (int a = 0; a < Q; ++a) {
                    size_t d = node_index(wrap(x + CV[a][0], nx), wrap(y + CV[a][1], ny),
                                          wrap(z + CV[a][2], nz), nx, ny);
                    nxt[(size_t)a * N + d] = fstar[a];
                }
            }
        }
        double *t = cur;
        cur = nxt;
        nxt = t;
    }
    if (cur != f) memcpy(f, cur, (size_t)Q * N * sizeof(double));
    free(psi);
    free(g);
    return 0;
}

/* Force field F (3*N, component-major) of the current state (Eq. 5). */
int orc_force(int nx, int ny, int nz, double G, int psi_form, double rho0, const double *f,
              double *F) {
    size_t N = (size_t)nx * ny * nz;
    double *psi = (double *)malloc(N * sizeof(double));
    if (!psi) return -1;
    psi_field(nx, ny, nz, psi_form, rho0, f, psi);
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                double Fl[3];
                node_force(nx, ny, nz, psi, x, y, z, G, Fl);
                size_t i = node_index(x, y, z, nx, ny);
                for (int k = 0; k < 3; ++k) F[(size_t)k * N + i] = Fl[k];
            }
    free(psi);
    return 0;
}

/*
 * Macroscopic fields: rho (Eq. 4) and the velocity of reading R7,
 * u = (j + F/2) / rho; bare != 0 gives u = j / rho instead.  Any output
 * pointer may be NULL.
 */
int orc_moments(int nx, int ny, int nz, double G, int psi_form, double rho0, const double *f,
                int bare, double *rho_out, double *ux, double *uy, double *uz) {
    size_t N = (size_t)nx * ny * nz;
    double *psi = (double *)malloc(N * sizeof(double));
    if (!psi) return -1;
    psi_field(nx, ny, nz, psi_form, rho0, f, psi);
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                size_t i = node_index(x, y, z, nx, ny);
                double rho, j[3], F[3] = {0.0, 0.0, 0.0};
                node_moments(f, N, i, &rho, j);
                if (!bare) node_force(nx, ny, nz, psi, x, y, z, G, F);
                if (rho_out) rho_out[i] = rho;
                if (ux) ux[i] = (j[0] + 0.5 * F[0]) / rho;
                if (uy) uy[i] = (j[1] + 0.5 * F[1]) / rho;
                if (uz) uz[i] = (j[2] + 0.5 * F[2]) / rho;
            }
    free(psi);
    return 0;
}

/* Radius of the perturbed ligament, R(x) = R0 (1 + eps cos(2 pi x / lambda + phase)). */
static double ligament_radius(int x, double R0, double lambda, double eps, double phase) {
    const double two_pi = 6.283185307179586476925286766559;
    return R0 * (1.0 + eps * cos(two_pi * (double)x / lambda + phase));
}

static double axis_distance(int y, int z, int ny, int nz) {
    double yc = 0.5 * (double)(ny - 1), zc = 0.5 * (double)(nz - 1); /* R12 */
    double dy = (double)y - yc, dz = (double)z - zc;
    return sqrt(dy * dy + dz * dz);
}

/*
 * Ligament initial condition (set-up section; perturbation in the
 * R0 (1 + eps cos(2 pi x / lambda + phase)) form, tanh interface R11,
 * f_a = w_a rho R13).
 */
void orc_init_ligament(int nx, int ny, int nz, double R0, double lambda, double eps,
                       double phase, double rho_l, double rho_v, double width, double *f) {
    size_t N = (size_t)nx * ny * nz;
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                double R = ligament_radius(x, R0, lambda, eps, phase);
                double r = axis_distance(y, z, ny, nz);
                double rho = rho_v + 0.5 * (rho_l - rho_v) * (1.0 - tanh(2.0 * (r - R) / width));
                size_t i = node_index(x, y, z, nx, ny);
                for (int a = 0; a < Q; ++a) f[(size_t)a * N + i] = WT[a] * rho;
            }
}

/*
 * Ligament initial condition through a tabulated radial profile (reading
 * R15): rho = prof(d), d = r - R(x) the signed distance to the interface,
 * prof sampled at d0 + k*dd (k = 0..n-1), linear interpolation, clamped at
 * both ends.
 */
void orc_init_profile(int nx, int ny, int nz, double R0, double lambda, double eps, double phase,
                      const double *prof, int n, double d0, double dd, double *f) {
    size_t N = (size_t)nx * ny * nz;
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                double d = axis_distance(y, z, ny, nz) - ligament_radius(x, R0, lambda, eps, phase);
                double s = (d - d0) / dd;
                double rho;
                if (s <= 0.0) {
                    rho = prof[0];
                } else if (s >= (double)(n - 1)) {
                    rho = prof[n - 1];
                } else {
                    int k = (int)floor(s);
                    double t = s - (double)k;
                    rho = prof[k] + t * (prof[k + 1] - prof[k]);
                }
                size_t i = node_index(x, y, z, nx, ny);
                for (int a = 0; a < Q; ++a) f[(size_t)a * N + i] = WT[a] * rho;
            }
}

/*
 * Connected components of a 0/1 mask, 6-connectivity, periodic in all three
 * directions, by breadth-first flood fill.  labels[i] = component number
 * (0..count-1, in order of the first node met in index order) or -1.
 * sizes (may be NULL) receives the node count of each component and must
 * hold N entries.  Returns the component count, or -1 on allocation failure.
 */
int orc_ccl(int nx, int ny, int nz, const unsigned char *mask, int *labels, long long *sizes) {
    size_t N = (size_t)nx * ny * nz;
    size_t *queue = (size_t *)malloc(N * sizeof(size_t));
    if (!queue) return -1;
    for (size_t i = 0; i < N; ++i) labels[i] = -1;
    int count = 0;
    static const int NB[6][3] = {{1, 0, 0}, {-1, 0, 0}, {0, 1, 0},
                                 {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};
    for (size_t s = 0; s < N; ++s) {
        if (!mask[s] || labels[s] >= 0) continue;
        size_t head = 0, tail = 0;
        queue[tail++] = s;
        labels[s] = count;
        long long members = 0;
        while (head < tail) {
            size_t i = queue[head++];
            ++members;
            int x = (int)(i % (size_t)nx);
            int y = (int)((i / (size_t)nx) % (size_t)ny);
            int z = (int)(i / ((size_t)nx * ny));
            for (int k = 0; k < 6; ++k) {
                size_t j = node_index(wrap(x + NB[k][0], nx), wrap(y + NB[k][1], ny),
                                      wrap(z + NB[k][2], nz), nx, ny);
                if (mask[j] && labels[j] < 0) {
                    labels[j] = count;
                    queue[tail++] = j;
                }
            }
        }
        if (sizes) sizes[count] = members;
        ++count;
    }
    free(queue);
    return count;
}

/*
 * Diagnostics of one state, plain sequential sums in index order.
 * Liquid: rho > (rho_l + rho_v)/2 (strict).  Weighted liquid fraction
 * phi = clamp((rho - rho_v)/(rho_l - rho_v), 0, 1).  Per x-slice liquid
 * area A(x) (count) and A_w(x) (sum of phi).
 * out[0] mass, out[1..3] total momentum sum_i j_i, out[4] liquid volume
 * sum phi, out[5] liquid count, out[6] min_x A_w(x), out[7] min_x A(x),
 * out[8] x of the minimum count (first), out[9] max |j/rho|,
 * out[10] min rho, out[11] max rho, out[12] 1 if every rho is finite and
 * positive else 0.
 * slice_w, slice_n (may be NULL): nx entries each.
 */
void orc_diagnostics(int nx, int ny, int nz, const double *f, double rho_l, double rho_v,
                     double *out, double *slice_w, double *slice_n) {
    size_t N = (size_t)nx * ny * nz;
    double thr = 0.5 * (rho_l + rho_v);
    double mass = 0.0, m[3] = {0.0, 0.0, 0.0}, vol = 0.0, cnt = 0.0, maxu = 0.0;
    double rmin = INFINITY, rmax = -INFINITY;
    int ok = 1;
    double *aw = (double *)calloc((size_t)nx, sizeof(double));
    double *an = (double *)calloc((size_t)nx, sizeof(double));
    for (size_t i = 0; i < N; ++i) {
        double rho, j[3];
        node_moments(f, N, i, &rho, j);
        int x = (int)(i % (size_t)nx);
        mass += rho;
        for (int k = 0; k < 3; ++k) m[k] += j[k];
        if (!(rho > 0.0) || !isfinite(rho)) ok = 0;
        if (rho < rmin) rmin = rho;
        if (rho > rmax) rmax = rho;
        double phi = (rho - rho_v) / (rho_l - rho_v);
        if (phi < 0.0) phi = 0.0;
        if (phi > 1.0) phi = 1.0;
        vol += phi;
        aw[x] += phi;
        if (rho > thr) {
            cnt += 1.0;
            an[x] += 1.0;
        }
        double u = sqrt(j[0] * j[0] + j[1] * j[1] + j[2] * j[2]) / rho;
        if (u > maxu) maxu = u;
    }
    double minw = INFINITY, minn = INFINITY;
    int minx = 0;
    for (int x = 0; x < nx; ++x) {
        if (aw[x] < minw) minw = aw[x];
        if (an[x] < minn) {
            minn = an[x];
            minx = x;
        }
        if (slice_w) slice_w[x] = aw[x];
        if (slice_n) slice_n[x] = an[x];
    }
    out[0] = mass;
    out[1] = m[0];
    out[2] = m[1];
    out[3] = m[2];
    out[4] = vol;
    out[5] = cnt;
    out[6] = minw;
    out[7] = minn;
    out[8] = (double)minx;
    out[9] = maxu;
    out[10] = rmin;
    out[11] = rmax;
    out[12] = (double)ok;
    free(aw);
    free(an);
}

/*
 * Droplet statistics (the droplets of the break-up study, reading R16/R17):
 * the liquid components of orc_ccl, each with
 *   first  smallest linear node index in the droplet,
 *   nodes  node count,
 *   vol    sum of phi = clamp((rho - rho_v)/(rho_l - rho_v), 0, 1),
 *   mass   sum of rho,
 *   c[3]   centroid of its nodes on the periodic box: per axis the circular
 *          mean, i.e. the direction of sum(cos t, sin t) with t = 2 pi x / n,
 *          mapped back to a coordinate in [0, n),
 *   r[3]   length of that mean vector divided by the node count (1 for a
 *          droplet in one plane, near 0 when the droplet fills the axis, in
 *          which case the centroid along it is not defined),
 *   xs     number of x slices holding a node of the droplet (nx: it wraps).
 * Records of ORC_DROPLET_REC doubles [first, nodes, vol, mass, c0, c1, c2,
 * r0, r1, r2, xs], sorted by node count (largest first), ties by first index.
 * Writes min(count, max_out) records; returns the droplet count, or -1 when
 * memory runs out.  Sums run in node-index order.
 */
#define ORC_DROPLET_REC 11
static int cmp_droplet(const void *pa, const void *pb) {
    const double *a = (const double *)pa, *b = (const double *)pb;
    if (a[1] != b[1]) return a[1] > b[1] ? -1 : 1;
    return a[0] < b[0] ? -1 : (a[0] > b[0] ? 1 : 0);
}

int orc_droplets(int nx, int ny, int nz, const double *f, double rho_l, double rho_v,
                 double *out, int max_out) {
    const double TWO_PI = 6.283185307179586476925286766559;
    size_t N = (size_t)nx * ny * nz;
    double thr = 0.5 * (rho_l + rho_v);
    double *rho = (double *)malloc(N * sizeof(double));
    unsigned char *mask = (unsigned char *)malloc(N);
    int *labels = (int *)malloc(N * sizeof(int));
    if (!rho || !mask || !labels) {
        free(rho); free(mask); free(labels);
        return -1;
    }
    for (size_t i = 0; i < N; ++i) {
        double j[3];
        node_moments(f, N, i, &rho[i], j);
        mask[i] = rho[i] > thr;
    }
    int count = orc_ccl(nx, ny, nz, mask, labels, NULL);
    /* per droplet: first, nodes, vol, mass, (cos, sin) x 3 */
    double *acc = count > 0 ? (double *)calloc((size_t)count * 10, sizeof(double)) : NULL;
    unsigned char *occ = count > 0 ? (unsigned char *)calloc((size_t)count * nx, 1) : NULL;
    if (count < 0 || (count > 0 && (!acc || !occ))) {
        free(rho); free(mask); free(labels); free(acc); free(occ);
        return -1;
    }
    for (int k = 0; k < count; ++k) acc[10 * k] = -1.0;
    const int dims[3] = {nx, ny, nz};
    for (size_t i = 0; i < N; ++i) {
        int k = labels[i];
        if (k < 0) continue;
        double *a = acc + 10 * (size_t)k;
        if (a[0] < 0.0) a[0] = (double)i;   /* the first node met in index order */
        int crd[3] = {(int)(i % (size_t)nx), (int)((i / (size_t)nx) % (size_t)ny),
                      (int)(i / ((size_t)nx * ny))};
        double phi = (rho[i] - rho_v) / (rho_l - rho_v);
        if (phi < 0.0) phi = 0.0;
        if (phi > 1.0) phi = 1.0;
        a[1] += 1.0;
        a[2] += phi;
        a[3] += rho[i];
        for (int d = 0; d < 3; ++d) {
            double t = TWO_PI * (double)crd[d] / (double)dims[d];
            a[4 + 2 * d] += cos(t);
            a[5 + 2 * d] += sin(t);
        }
        occ[(size_t)k * nx + crd[0]] = 1;
    }
    double *rec = count > 0 ? (double *)malloc((size_t)count * ORC_DROPLET_REC * sizeof(double)) : NULL;
    if (count > 0 && !rec) {
        free(rho); free(mask); free(labels); free(acc); free(occ);
        return -1;
    }
    for (int k = 0; k < count; ++k) {
        const double *a = acc + 10 * (size_t)k;
        double *r = rec + (size_t)k * ORC_DROPLET_REC;
        r[0] = a[0];
        r[1] = a[1];
        r[2] = a[2];
        r[3] = a[3];
        for (int d = 0; d < 3; ++d) {
            double c = a[4 + 2 * d], sn = a[5 + 2 * d];
            double t = atan2(sn, c);
            if (t < 0.0) t += TWO_PI;
            double pos = t / TWO_PI * (double)dims[d];
            if (pos >= (double)dims[d]) pos -= (double)dims[d];
            r[4 + d] = pos;
            r[7 + d] = sqrt(c * c + sn * sn) / a[1];
        }
        int xs = 0;
        for (int x = 0; x < nx; ++x) xs += occ[(size_t)k * nx + x];
        r[10] = (double)xs;
    }
    if (count > 1) qsort(rec, (size_t)count, ORC_DROPLET_REC * sizeof(double), cmp_droplet);
    int n = count < max_out ? count : max_out;
    if (n > 0) memcpy(out, rec, (size_t)n * ORC_DROPLET_REC * sizeof(double));
    free(rho); free(mask); free(labels); free(acc); free(occ); free(rec);
    return count;
}

/*
 * One time step evaluated only at selected nodes: out[k*19 + a] is the
 * population a at node nodes[k] after the step, i.e. the post-collision
 * value of the upstream node nodes[k] - c_a.  psi is evaluated on demand,
 * so the cost per node is independent of the lattice size.
 */
void orc_step_nodes(int nx, int ny, int nz, double tau, double G, int psi_form, double rho0,
                    const double *f, const long long *nodes, int count, double *out) {
    size_t N = (size_t)nx * ny * nz;
#pragma omp parallel for schedule(dynamic, 16)
    for (int k = 0; k < count; ++k) {
        size_t i = (size_t)nodes[k];
        int x = (int)(i % (size_t)nx);
        int y = (int)((i / (size_t)nx) % (size_t)ny);
        int z = (int)(i / ((size_t)nx * ny));
        for (int a = 0; a < Q; ++a) {
            int sx = wrap(x - CV[a][0], nx), sy = wrap(y - CV[a][1], ny), sz = wrap(z - CV[a][2], nz);
            size_t si = node_index(sx, sy, sz, nx, ny);
            double rho, j[3], s[3] = {0.0, 0.0, 0.0};
            node_moments(f, N, si, &rho, j);
            for (int b = 0; b < Q; ++b) {
                size_t nb = node_index(wrap(sx + CV[b][0], nx), wrap(sy + CV[b][1], ny),
                                       wrap(sz + CV[b][2], nz), nx, ny);
                double rn, jn[3];
                node_moments(f, N, nb, &rn, jn);
                double pn = orc_psi(rn, psi_form, rho0);
                for (int c = 0; c < 3; ++c) s[c] += WT[b] * pn * CV[b][c];
            }
            double p = orc_psi(rho, psi_form, rho0);
            double F[3], u[3], feq[Q];
            for (int c = 0; c < 3; ++c) F[c] = -G * p * s[c];
            for (int c = 0; c < 3; ++c) u[c] = j[c] / rho + F[c] * tau / rho;
            orc_feq(rho, u, feq);
            double fa = f[(size_t)a * N + si];
            out[(size_t)k * Q + a] = fa - (fa - feq[a]) / tau;
        }
    }
}

/*
 * Flat-interface coexistence run (reading R14): a liquid slab across x in
 * a periodic n x 3 x 3 box.  When init != 0 the slab is set up here with a
 * tanh profile between rho_l0 and rho_v0 on [n/4, 3n/4); when init == 0, f
 * must already hold a state (used to continue a converged run to another
 * tau).  Runs blocks of
 * `check` steps until max |rho(t) - rho(t - check)| < tol or max_steps.
 * out[0] = rho at the slab centre x = n/2, out[1] = rho at x = 0,
 * out[2] = steps run, out[3] = last max |drho|.  prof (may be NULL): the
 * n densities along x of the final state.  f (19 * n * 9) holds the final
 * state.  rates != NULL runs the MRT collision with those 19 rates instead
 * of the paper's SRT step (tau is then unused).
 */
int orc_coexistence_ex(int n, double tau, const double *rates, double G, int psi_form, double rho0,
                       double rho_l0, double rho_v0, int init, double tol, int check,
                       long long max_steps, double *f, double *out, double *prof) {
    const int ny = 3, nz = 3;
    size_t N = (size_t)n * ny * nz;
    double *rprev = (double *)malloc(N * sizeof(double));
    if (!rprev) return -1;
    if (init) {
        for (int z = 0; z < nz; ++z)
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < n; ++x) {
                    double x1 = 0.25 * n, x2 = 0.75 * n;
                    double rho = rho_v0 + 0.5 * (rho_l0 - rho_v0) *
                                              (tanh((double)x - x1) - tanh((double)x - x2));
                    size_t i = node_index(x, y, z, n, ny);
                    for (int a = 0; a < Q; ++a) f[(size_t)a * N + i] = WT[a] * rho;
                }
    }
    long long steps = 0;
    double dmax = INFINITY;
    for (size_t i = 0; i < N; ++i) {
        double j[3];
        node_moments(f, N, i, &rprev[i], j);
    }
    while (steps < max_steps) {
        int rc = rates ? orc_step_forcing(n, ny, nz, tau, rates, G, psi_form, rho0, f, check)
                       : orc_step(n, ny, nz, tau, G, psi_form, rho0, f, check);
        if (rc != 0) {
            free(rprev);
            return -1;
        }
        steps += check;
        dmax = 0.0;
        int bad = 0;
        for (size_t i = 0; i < N; ++i) {
            double rho, j[3];
            node_moments(f, N, i, &rho, j);
            if (!isfinite(rho)) bad = 1;
            double d = fabs(rho - rprev[i]);
            if (d > dmax) dmax = d;
            rprev[i] = rho;
        }
        if (bad) {
            dmax = NAN;
            break;
        }
        if (dmax < tol) break;
    }
    out[0] = rprev[node_index(n / 2, 1, 1, n, ny)];
    out[1] = rprev[node_index(0, 1, 1, n, ny)];
    out[2] = (double)steps;
    out[3] = dmax;
    if (prof)
        for (int x = 0; x < n; ++x) prof[x] = rprev[node_index(x, 1, 1, n, ny)];
    free(rprev);
    return 0;
}

/* Flat-interface run of the paper's SRT model (orc_coexistence_ex with no
 * MRT rates). */
int orc_coexistence(int n, double tau, double G, int psi_form, double rho0, double rho_l0,
                    double rho_v0, int init, double tol, int check, long long max_steps,
                    double *f, double *out, double *prof) {
    return orc_coexistence_ex(n, tau, NULL, G, psi_form, rho0, rho_l0, rho_v0, init, tol, check,
                              max_steps, f, out, prof);
}
