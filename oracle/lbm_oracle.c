/*
 * lbm_oracle.c -- plain, slow FP64 CPU oracle of the He-Luo MRT lattice Boltzmann step
 * with the strain-rate tensor formed by both of the paper's routes (Zhang, Huang, Wang, Shi,
 * "The computation of strain rate tensor in multiple-relaxation-time lattice Boltzmann model",
 * arXiv:1704.07559).
 *
 * TEST INFRASTRUCTURE ONLY.  The product (the CUDA library) never links, loads or calls this
 * file.  Only the test suite, the smoke check and the CPU-baseline leg of the benchmark use it.
 * It shares no code, header or table with the CUDA path: every table here is typed in from
 * the paper (D3Q19) or from the textbook definition stated beside it (D2Q9).
 *
 * Everything is written literally: dense q x q matrices where the paper has matrices, one node
 * at a time, no fusion and no reordering.  T^-1 is obtained by Gauss-Jordan elimination of the
 * printed T (not by the orthogonality shortcut), so the tests can compare the two.
 *
 * Paper passages followed (sections and equations of the paper):
 *   Sec. 2   eq. (edf)        He-Luo equilibrium in delta-rho form
 *            eq. (omega)      weights;  eq. (HeLuoD3Q19) velocity set
 *            matrix T         d'Humieres 19x19 moment matrix
 *            eq. (mrteqvT)    collision in moment space, f* = f - T^-1 L (m - m_eq)
 *            eq. (meq)        equilibrium moments, w_eps = 3, w_epsj = -11/2, w_xx = -1/2
 *            eq. (sD3Q15)     diagonal rates, s_0 = s_3 = s_5 = s_7 = 0
 *   Sec. 3   eq. (LuoS)       Yu formula, S from 6 non-equilibrium moments
 *            eq. (ChaiS)      Chai formula, S from the 19 non-equilibrium distributions
 *   Sec. 4.1 eq. (YuLuobasis) first-order non-equilibrium moments in terms of grad j
 *            (used to initialise a state whose strain rate is a given velocity gradient)
 *   Sec. 5.4 the Chai-based procedure for a Yu-type formula on another lattice (D2Q9, D3Q15)
 *
 * Readings where the paper is silent (each one is listed with its reason in the design notes):
 *   - D2Q9 lattice and moment basis: the Lallemand-Luo basis (paper names D2Q9 only).
 *   - D3Q15 lattice and moment basis: the d'Humieres et al. (2002) 15-moment basis (paper
 *     names D3Q15 only), equilibrium moments = T f_eq of the same He-Luo equilibrium.
 *   - Force: Guo-type discrete force Fbar_i = w_i[(c_i-u)/cs2 + (c_i.u)c_i/cs4].F, collision
 *     source (I - L/2) T Fbar, j = sum c f + F/2, and both strain formulas use the effective
 *     non-equilibrium (f - f_eq + Fbar/2).
 *   - Closures: Smagorinsky tau = tau0 + 3 Cs^2 |S|, power law tau = 1/2 + 3 K |S|^(n-1)
 *     clamped, |S| = sqrt(2 S:S); both solved per node by fixed-point iteration on tau with
 *     S recomputed from the same pre-collision state.  Two Smagorinsky variants: lagged (the
 *     collision uses the tau that the previous step stored at the node, and stores
 *     tau0 + 3 Cs^2 |S| for the next one) and deviatoric (tau = tau0 + 3 Cs^2 |S_d| with S_d the
 *     traceless part of S, solved to convergence).
 *   - Boundaries: periodic, halfway bounce-back wall, moving wall (Ladd momentum term).
 *   - Viscosity: nu = (tau - 1/2)/3.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_ERR_ARG -1

#define BC_PERIODIC 0
#define BC_WALL 1
#define BC_LID 2

#define CL_NEWTON 0
#define CL_SMAG 1
#define CL_POWERLAW 2
#define CL_SMAG_LAGGED 3
#define CL_SMAG_DEV 4

#define F_YU 0
#define F_CHAI 1

/* ------------------------------------------------------------------------------------------ */
/* Lattice tables                                                                              */
/* ------------------------------------------------------------------------------------------ */

/* D3Q19 velocities, eq. (HeLuoD3Q19): the three printed rows read column by column. */
static const int C19[19][3] = {
    {0, 0, 0},   {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},  {0, 0, -1},
    {1, 1, 0},   {-1, 1, 0}, {1, -1, 0}, {-1, -1, 0}, {1, 0, 1}, {-1, 0, 1}, {1, 0, -1},
    {-1, 0, -1}, {0, 1, 1},  {0, -1, 1}, {0, 1, -1}, {0, -1, -1}};

/* D3Q19 moment matrix T as printed in Sec. 2 (d'Humieres basis), row by row. */
static const int T19[19][19] = {
    {1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1},
    {-30, -11, -11, -11, -11, -11, -11, 8, 8, 8, 8, 8, 8, 8, 8, 8, 8, 8, 8},
    {12, -4, -4, -4, -4, -4, -4, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1},
    {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0},
    {0, -4, 4, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0},
    {0, 0, 0, 1, -1, 0, 0, 1, 1, -1, -1, 0, 0, 0, 0, 1, -1, 1, -1},
    {0, 0, 0, -4, 4, 0, 0, 1, 1, -1, -1, 0, 0, 0, 0, 1, -1, 1, -1},
    {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1},
    {0, 0, 0, 0, 0, -4, 4, 0, 0, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1},
    {0, 2, 2, -1, -1, -1, -1, 1, 1, 1, 1, 1, 1, 1, 1, -2, -2, -2, -2},
    {0, -4, -4, 2, 2, 2, 2, 1, 1, 1, 1, 1, 1, 1, 1, -2, -2, -2, -2},
    {0, 0, 0, 1, 1, -1, -1, 1, 1, 1, 1, -1, -1, -1, -1, 0, 0, 0, 0},
    {0, 0, 0, -2, -2, 2, 2, 1, 1, 1, 1, -1, -1, -1, -1, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, -1, -1, 1},
    {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 0, 0, 1, -1, 1, -1, -1, 1, -1, 1, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 0, 0, -1, -1, 1, 1, 0, 0, 0, 0, 1, -1, 1, -1},
    {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 1, -1, -1, -1, -1, 1, 1}};

/* D2Q9: the paper names this lattice but does not print it.  Velocity order: rest, the four
 * axis directions counter-clockwise from +x, the four diagonals counter-clockwise from (1,1). */
static const int C9[9][3] = {{0, 0, 0},  {1, 0, 0},   {0, 1, 0},  {-1, 0, 0}, {0, -1, 0},
                             {1, 1, 0},  {-1, 1, 0},  {-1, -1, 0}, {1, -1, 0}};

/* D2Q9 moment matrix (Lallemand-Luo basis), rows are the polynomials
 * 1, e = -4 + 3c^2, eps = 4 - 21c^2/2 + 9c^4/2, j_x = c_x, q_x = (-5 + 3c^2) c_x,
 * j_y = c_y, q_y = (-5 + 3c^2) c_y, p_xx = c_x^2 - c_y^2, p_xy = c_x c_y, evaluated at C9. */
static const int T9[9][9] = {{1, 1, 1, 1, 1, 1, 1, 1, 1},    {-4, -1, -1, -1, -1, 2, 2, 2, 2},
                             {4, -2, -2, -2, -2, 1, 1, 1, 1},  {0, 1, 0, -1, 0, 1, -1, -1, 1},
                             {0, -2, 0, 2, 0, 1, -1, -1, 1},   {0, 0, 1, 0, -1, 1, 1, -1, -1},
                             {0, 0, -2, 0, 2, 1, 1, -1, -1},   {0, 1, -1, 1, -1, 0, 0, 0, 0},
                             {0, 0, 0, 0, 0, 1, -1, 1, -1}};

/* D3Q15: the paper names this lattice but does not print it.  Velocity order: rest, +x, -x, +y,
 * -y, +z, -z, then the eight corners (+-1, +-1, +-1) with c_x alternating fastest, then c_y,
 * then c_z (first (1,1,1), last (-1,-1,-1)). */
static const int C15[15][3] = {{0, 0, 0},  {1, 0, 0},   {-1, 0, 0},  {0, 1, 0},  {0, -1, 0},
                               {0, 0, 1},  {0, 0, -1},  {1, 1, 1},   {-1, 1, 1}, {1, -1, 1},
                               {-1, -1, 1}, {1, 1, -1}, {-1, 1, -1}, {1, -1, -1}, {-1, -1, -1}};

/* D3Q15 moment matrix (d'Humieres et al. 2002 basis), rows are the polynomials
 * 1, e = c^2 - 2, eps = (15c^4 - 55c^2 + 32)/2, j_x, q_x = (5c^2 - 13) c_x / 2, j_y, q_y, j_z, q_z,
 * 3p_xx = 3c_x^2 - c^2, p_ww = c_y^2 - c_z^2, p_xy = c_x c_y, p_yz = c_y c_z, p_xz = c_x c_z,
 * m_xyz = c_x c_y c_z, evaluated at C15. */
static const int T15[15][15] = {
    {1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1},
    {-2, -1, -1, -1, -1, -1, -1, 1, 1, 1, 1, 1, 1, 1, 1},
    {16, -4, -4, -4, -4, -4, -4, 1, 1, 1, 1, 1, 1, 1, 1},
    {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1},
    {0, -4, 4, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1},
    {0, 0, 0, 1, -1, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1},
    {0, 0, 0, -4, 4, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1},
    {0, 0, 0, 0, 0, 1, -1, 1, 1, 1, 1, -1, -1, -1, -1},
    {0, 0, 0, 0, 0, -4, 4, 1, 1, 1, 1, -1, -1, -1, -1},
    {0, 2, 2, -1, -1, -1, -1, 0, 0, 0, 0, 0, 0, 0, 0},
    {0, 0, 0, 1, 1, -1, -1, 0, 0, 0, 0, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1},
    {0, 0, 0, 0, 0, 0, 0, 1, 1, -1, -1, -1, -1, 1, 1},
    {0, 0, 0, 0, 0, 0, 0, 1, -1, 1, -1, -1, 1, -1, 1},
    {0, 0, 0, 0, 0, 0, 0, 1, -1, -1, 1, -1, 1, 1, -1}};

typedef struct {
    int q, d;
    int c[19][3];
    double w[19];
    double T[19][19];
    double Tinv[19][19];
    int opp[19];
    int nu_idx[5]; /* moments relaxed with s_nu (the viscous stresses) */
    int n_nu;
} lattice_t;

static lattice_t LAT19, LAT15, LAT9;
static int lat_ready = 0;

/* Gauss-Jordan inverse with partial pivoting, n <= 19.  Returns 0 on success. */
static int invert(int n, const double A[19][19], double Ainv[19][19]) {
    double M[19][38];
    for (int r = 0; r < n; ++r) {
        for (int k = 0; k < n; ++k) {
            M[r][k] = A[r][k];
            M[r][n + k] = (r == k) ? 1.0 : 0.0;
        }
    }
    for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int r = col + 1; r < n; ++r)
            if (fabs(M[r][col]) > fabs(M[piv][col])) piv = r;
        if (M[piv][col] == 0.0) return -1;
        if (piv != col)
            for (int k = 0; k < 2 * n; ++k) {
                double t = M[col][k];
                M[col][k] = M[piv][k];
                M[piv][k] = t;
            }
        double inv = 1.0 / M[col][col];
        for (int k = 0; k < 2 * n; ++k) M[col][k] *= inv;
        for (int r = 0; r < n; ++r) {
            if (r == col || M[r][col] == 0.0) continue;
            double fct = M[r][col];
            for (int k = 0; k < 2 * n; ++k) M[r][k] -= fct * M[col][k];
        }
    }
    for (int r = 0; r < n; ++r)
        for (int k = 0; k < n; ++k) Ainv[r][k] = M[r][n + k];
    return 0;
}

static void setup_lattice(lattice_t *L, int q) {
    memset(L, 0, sizeof(*L));
    L->q = q;
    if (q == 19) {
        L->d = 3;
        for (int i = 0; i < 19; ++i) {
            for (int a = 0; a < 3; ++a) L->c[i][a] = C19[i][a];
            for (int k = 0; k < 19; ++k) L->T[i][k] = T19[i][k];
        }
        /* eq. (omega): 1/3 rest, 1/18 axis (i = 1..6), 1/36 edges (i = 7..18) */
        for (int i = 0; i < 19; ++i) L->w[i] = (i == 0) ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
        /* eq. (sD3Q15meaning): s_nu relaxes moments 9, 11, 13, 14, 15 */
        int nu[5] = {9, 11, 13, 14, 15};
        for (int k = 0; k < 5; ++k) L->nu_idx[k] = nu[k];
        L->n_nu = 5;
    } else if (q == 15) {
        L->d = 3;
        for (int i = 0; i < 15; ++i) {
            for (int a = 0; a < 3; ++a) L->c[i][a] = C15[i][a];
            for (int k = 0; k < 15; ++k) L->T[i][k] = T15[i][k];
        }
        /* 2/9 rest, 1/9 axis (i = 1..6), 1/72 corners (i = 7..14) */
        for (int i = 0; i < 15; ++i) L->w[i] = (i == 0) ? 2.0 / 9.0 : (i <= 6 ? 1.0 / 9.0 : 1.0 / 72.0);
        /* s_nu relaxes the five viscous stresses 3p_xx, p_ww, p_xy, p_yz, p_xz (moments 9..13) */
        for (int k = 0; k < 5; ++k) L->nu_idx[k] = 9 + k;
        L->n_nu = 5;
    } else {
        L->d = 2;
        for (int i = 0; i < 9; ++i) {
            for (int a = 0; a < 3; ++a) L->c[i][a] = C9[i][a];
            for (int k = 0; k < 9; ++k) L->T[i][k] = T9[i][k];
        }
        for (int i = 0; i < 9; ++i) L->w[i] = (i == 0) ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
        L->nu_idx[0] = 7;
        L->nu_idx[1] = 8;
        L->n_nu = 2;
    }
    invert(q, (const double(*)[19])L->T, L->Tinv);
    for (int i = 0; i < q; ++i)
        for (int k = 0; k < q; ++k)
            if (L->c[k][0] == -L->c[i][0] && L->c[k][1] == -L->c[i][1] && L->c[k][2] == -L->c[i][2])
                L->opp[i] = k;
}

static const lattice_t *lattice(int q) {
    if (!lat_ready) {
        setup_lattice(&LAT19, 19);
        setup_lattice(&LAT15, 15);
        setup_lattice(&LAT9, 9);
        lat_ready = 1;
    }
    if (q == 19) return &LAT19;
    if (q == 15) return &LAT15;
    if (q == 9) return &LAT9;
    return NULL;
}

/* Export the tables: c (q x 3 ints), w (q), T (q x q), Tinv (q x q, by elimination), opp (q). */
int or_tables(int q, int *c, double *w, double *T, double *Tinv, int *opp) {
    const lattice_t *L = lattice(q);
    if (!L) return OR_ERR_ARG;
    for (int i = 0; i < q; ++i) {
        if (c)
            for (int a = 0; a < 3; ++a) c[3 * i + a] = L->c[i][a];
        if (w) w[i] = L->w[i];
        if (opp) opp[i] = L->opp[i];
        for (int k = 0; k < q; ++k) {
            if (T) T[q * i + k] = L->T[i][k];
            if (Tinv) Tinv[q * i + k] = L->Tinv[i][k];
        }
    }
    return OR_OK;
}

/* ------------------------------------------------------------------------------------------ */
/* Equilibria, force, strain rate                                                              */
/* ------------------------------------------------------------------------------------------ */

static const double CS2 = 1.0 / 3.0;

/* eq. (edf), delta-rho form:  f_i^eq = w_i [drho + rho0 (c.u/cs2 + (c.u)^2/(2 cs4) - u^2/(2 cs2))],
 * with u = j / rho0. */
int or_feq(int q, double drho, const double *j, double rho0, double *feq) {
    const lattice_t *L = lattice(q);
    if (!L) return OR_ERR_ARG;
    double u[3] = {j[0] / rho0, j[1] / rho0, L->d == 3 ? j[2] / rho0 : 0.0};
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < q; ++i) {
        double cu = L->c[i][0] * u[0] + L->c[i][1] * u[1] + L->c[i][2] * u[2];
        feq[i] = L->w[i] * (drho + rho0 * (cu / CS2 + cu * cu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2)));
    }
    return OR_OK;
}

/* Equilibrium moments in closed form.
 * D3Q19: eq. (meq) with w_eps = 3, w_epsj = -11/2, w_xx = -1/2.  The labels of the p_xx/pi_xx
 * lines in the printed set are read so that moment 9 = 3p_xx, 10 = 3pi_xx, 11 = p_ww and
 * 12 = pi_ww follow the moment vector eq. (moment) and the first row-block of eq. (solvem).
 * D2Q9 (Lallemand-Luo basis with the He-Luo equilibrium):
 *   (drho, -2 drho + 3 j^2/rho0, drho - 3 j^2/rho0, jx, -jx, jy, -jy, (jx^2 - jy^2)/rho0, jx jy/rho0).
 * D3Q15 (d'Humieres basis with the He-Luo equilibrium, i.e. T f_eq worked out by hand):
 *   (drho, -drho + j^2/rho0, drho - 5 j^2/rho0, jx, -7jx/3, jy, -7jy/3, jz, -7jz/3,
 *    (3jx^2 - j^2)/rho0, (jy^2 - jz^2)/rho0, jx jy/rho0, jy jz/rho0, jx jz/rho0, 0). */
int or_meq(int q, double drho, const double *j, double rho0, double *meq) {
    if (q == 19) {
        const double w_eps = 3.0, w_epsj = -11.0 / 2.0, w_xx = -1.0 / 2.0;
        double jx = j[0], jy = j[1], jz = j[2];
        double jj = jx * jx + jy * jy + jz * jz;
        meq[0] = drho;
        meq[1] = -11.0 * drho + 19.0 / rho0 * jj;
        meq[2] = w_eps * drho + w_epsj / rho0 * jj;
        meq[3] = jx;
        meq[4] = -2.0 * jx / 3.0;
        meq[5] = jy;
        meq[6] = -2.0 * jy / 3.0;
        meq[7] = jz;
        meq[8] = -2.0 * jz / 3.0;
        meq[9] = (3.0 * jx * jx - jj) / rho0; /* 3 p_xx */
        meq[10] = w_xx * meq[9];              /* 3 pi_xx = 3 w_xx p_xx */
        meq[11] = (jy * jy - jz * jz) / rho0; /* p_ww */
        meq[12] = w_xx * meq[11];             /* pi_ww = w_xx p_ww */
        meq[13] = jx * jy / rho0;
        meq[14] = jy * jz / rho0;
        meq[15] = jx * jz / rho0;
        meq[16] = 0.0;
        meq[17] = 0.0;
        meq[18] = 0.0;
        return OR_OK;
    }
    if (q == 15) {
        double jx = j[0], jy = j[1], jz = j[2];
        double jj = jx * jx + jy * jy + jz * jz;
        meq[0] = drho;
        meq[1] = -drho + jj / rho0;
        meq[2] = drho - 5.0 * jj / rho0;
        meq[3] = jx;
        meq[4] = -7.0 * jx / 3.0;
        meq[5] = jy;
        meq[6] = -7.0 * jy / 3.0;
        meq[7] = jz;
        meq[8] = -7.0 * jz / 3.0;
        meq[9] = (3.0 * jx * jx - jj) / rho0;
        meq[10] = (jy * jy - jz * jz) / rho0;
        meq[11] = jx * jy / rho0;
        meq[12] = jy * jz / rho0;
        meq[13] = jx * jz / rho0;
        meq[14] = 0.0;
        return OR_OK;
    }
    if (q == 9) {
        double jx = j[0], jy = j[1];
        double jj = jx * jx + jy * jy;
        meq[0] = drho;
        meq[1] = -2.0 * drho + 3.0 * jj / rho0;
        meq[2] = drho - 3.0 * jj / rho0;
        meq[3] = jx;
        meq[4] = -jx;
        meq[5] = jy;
        meq[6] = -jy;
        meq[7] = (jx * jx - jy * jy) / rho0;
        meq[8] = jx * jy / rho0;
        return OR_OK;
    }
    return OR_ERR_ARG;
}

/* Guo-type discrete force (reading; the paper cites forced MRT only by reference):
 * Fbar_i = w_i [ (c_i - u) . F / cs2 + (c_i . u)(c_i . F) / cs4 ],  u = j / rho0. */
int or_force_bar(int q, const double *j, double rho0, const double *F, double *Fbar) {
    const lattice_t *L = lattice(q);
    if (!L) return OR_ERR_ARG;
    double u[3] = {j[0] / rho0, j[1] / rho0, L->d == 3 ? j[2] / rho0 : 0.0};
    double Fv[3] = {F[0], F[1], L->d == 3 ? F[2] : 0.0};
    for (int i = 0; i < q; ++i) {
        double cmuF = 0.0, cu = 0.0, cF = 0.0;
        for (int a = 0; a < 3; ++a) {
            cmuF += (L->c[i][a] - u[a]) * Fv[a];
            cu += L->c[i][a] * u[a];
            cF += L->c[i][a] * Fv[a];
        }
        Fbar[i] = L->w[i] * (cmuF / CS2 + cu * cF / (CS2 * CS2));
    }
    return OR_OK;
}

/* Number of strain-rate components stored: 6 in 3D (xx, yy, zz, xy, yz, xz), 3 in 2D (xx, yy, xy). */
static int n_strain(int q) { return q == 9 ? 3 : 6; }

/* Yu formula, eq. (LuoS), written as printed (delta_t = 1, eps m^(1) = m - m_eq).
 * s holds all q rates; the formula reads s_1 and s_9 (it assumes s_9 = s_11 = s_13..15).
 * D2Q9: the Yu-type formula obtained by the Sec. 5.4 procedure from Chai's formula:
 *   S_xx,yy = -(s_e m_e +- 3 s_nu m_pxx) / (4 rho0),  S_xy = -3 s_nu m_pxy / (2 rho0).
 * D3Q15: the same procedure (S = -3/(2 rho0) sum_i c_i c_i [T^-1 L m_neq]_i with the d'Humieres
 * basis) gives
 *   S_xx = -(s_e m_e + s_nu m_3pxx) / (2 rho0),
 *   S_yy,zz = -(2 s_e m_e - s_nu m_3pxx +- 3 s_nu m_pww) / (4 rho0),
 *   S_xy = -3 s_nu m_pxy / (2 rho0),  S_yz = -3 s_nu m_pyz / (2 rho0),  S_xz = -3 s_nu m_pxz / (2 rho0). */
int or_strain_yu(int q, const double *mneq, const double *s, double rho0, double *S) {
    if (q == 19) {
        double m1 = mneq[1], m9 = mneq[9], m11 = mneq[11];
        double s1 = s[1], s9 = s[9];
        S[0] = -(s1 * m1 + 19.0 * s9 * m9) / (38.0 * rho0);
        S[1] = -(2.0 * s1 * m1 - 19.0 * s9 * (m9 - 3.0 * m11)) / (76.0 * rho0);
        S[2] = -(2.0 * s1 * m1 - 19.0 * s9 * (m9 + 3.0 * m11)) / (76.0 * rho0);
        S[3] = -3.0 * s9 * mneq[13] / (2.0 * rho0); /* xy */
        S[4] = -3.0 * s9 * mneq[14] / (2.0 * rho0); /* yz */
        S[5] = -3.0 * s9 * mneq[15] / (2.0 * rho0); /* zx */
        return OR_OK;
    }
    if (q == 15) {
        double se = s[1], snu = s[9];
        double e = se * mneq[1], p = snu * mneq[9], w = snu * mneq[10];
        S[0] = -(e + p) / (2.0 * rho0);
        S[1] = -(2.0 * e - p + 3.0 * w) / (4.0 * rho0);
        S[2] = -(2.0 * e - p - 3.0 * w) / (4.0 * rho0);
        S[3] = -3.0 * snu * mneq[11] / (2.0 * rho0); /* xy */
        S[4] = -3.0 * snu * mneq[12] / (2.0 * rho0); /* yz */
        S[5] = -3.0 * snu * mneq[13] / (2.0 * rho0); /* zx */
        return OR_OK;
    }
    if (q == 9) {
        double se = s[1], snu = s[7];
        S[0] = -(se * mneq[1] + 3.0 * snu * mneq[7]) / (4.0 * rho0);
        S[1] = -(se * mneq[1] - 3.0 * snu * mneq[7]) / (4.0 * rho0);
        S[2] = -3.0 * snu * mneq[8] / (2.0 * rho0);
        return OR_OK;
    }
    return OR_ERR_ARG;
}

/* Chai formula, eq. (ChaiS):  S = - sum_i c_i c_i (T^-1 L T)_ij f_j^neq / (2 rho0 cs2 delta_t),
 * computed literally: the dense q x q product T^-1 diag(s) T, applied to f^neq, then the second
 * velocity moment. */
int or_strain_chai(int q, const double *fneq, const double *s, double rho0, double *S) {
    const lattice_t *L = lattice(q);
    if (!L) return OR_ERR_ARG;
    double K[19][19];
    for (int i = 0; i < q; ++i)
        for (int j = 0; j < q; ++j) {
            double acc = 0.0;
            for (int k = 0; k < q; ++k) acc += L->Tinv[i][k] * s[k] * L->T[k][j];
            K[i][j] = acc;
        }
    double M[19];
    for (int i = 0; i < q; ++i) {
        double acc = 0.0;
        for (int j = 0; j < q; ++j) acc += K[i][j] * fneq[j];
        M[i] = acc;
    }
    static const int ab3[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {1, 2}, {0, 2}};
    static const int ab2[3][2] = {{0, 0}, {1, 1}, {0, 1}};
    int ns = n_strain(q);
    for (int p = 0; p < ns; ++p) {
        int a = (L->d == 3) ? ab3[p][0] : ab2[p][0];
        int b = (L->d == 3) ? ab3[p][1] : ab2[p][1];
        double N = 0.0;
        for (int i = 0; i < q; ++i) N += L->c[i][a] * L->c[i][b] * M[i];
        S[p] = -N / (2.0 * rho0 * CS2);
    }
    return OR_OK;
}

/* ------------------------------------------------------------------------------------------ */
/* Parameters, closure and the per-node collision                                              */
/* ------------------------------------------------------------------------------------------ */

typedef struct {
    int q;            /* 9, 15 or 19 */
    int closure;      /* CL_NEWTON, CL_SMAG, CL_POWERLAW */
    int formula;      /* F_YU or F_CHAI: the route whose S feeds the closure */
    int smag_iters;   /* fixed number of fixed-point sweeps for Smagorinsky */
    int pl_max_iter;  /* cap on power-law fixed-point sweeps */
    int bc[6];        /* faces -x, +x, -y, +y, -z, +z: BC_PERIODIC, BC_WALL, BC_LID */
    double rho0;
    double s[19];     /* relaxation rates; the s_nu entries hold 1/tau0 */
    double smag_cs;   /* Smagorinsky constant (filter width 1) */
    double pl_n, pl_k, pl_tau_min, pl_tau_max, pl_tol;
    double lid_u[6][3];
} or_params;

static int strain_components(int q) { return n_strain(q); }

static double strain_norm(int q, const double *S) {
    /* |S| = sqrt(2 S:S) */
    double ss;
    if (q != 9)
        ss = S[0] * S[0] + S[1] * S[1] + S[2] * S[2] + 2.0 * (S[3] * S[3] + S[4] * S[4] + S[5] * S[5]);
    else
        ss = S[0] * S[0] + S[1] * S[1] + 2.0 * S[2] * S[2];
    return sqrt(2.0 * ss);
}

/* |S_d| = sqrt(2 S_d:S_d), S_d = S - tr(S)/d I (the traceless part). */
static double dev_norm(int q, const double *S) {
    double ss;
    if (q != 9) {
        double t = (S[0] + S[1] + S[2]) / 3.0;
        double a = S[0] - t, b = S[1] - t, c = S[2] - t;
        ss = a * a + b * b + c * c + 2.0 * (S[3] * S[3] + S[4] * S[4] + S[5] * S[5]);
    } else {
        double t = (S[0] + S[1]) / 2.0;
        double a = S[0] - t, b = S[1] - t;
        ss = a * a + b * b + 2.0 * S[2] * S[2];
    }
    return sqrt(2.0 * ss);
}

/* S of the current node for a given s_nu (all s_nu entries set to snu), by the chosen route.
 * mneq: effective non-equilibrium moments; fneq: effective non-equilibrium distributions. */
static void strain_at(const or_params *p, const lattice_t *L, const double *mneq, const double *fneq,
                      double snu, double *S) {
    double s[19];
    for (int k = 0; k < L->q; ++k) s[k] = p->s[k];
    for (int k = 0; k < L->n_nu; ++k) s[L->nu_idx[k]] = snu;
    if (p->formula == F_YU)
        or_strain_yu(L->q, mneq, s, p->rho0, S);
    else
        or_strain_chai(L->q, fneq, s, p->rho0, S);
}

/* Solve the closure for tau at one node; returns the number of sweeps taken.
 * tau_prev: the tau stored at the node by the previous step (read by the lagged closure only);
 * *tau_next: the tau to store for the next step (lagged: tau0 + 3 Cs^2 |S|; others: tau). */
static int solve_tau(const or_params *p, const lattice_t *L, const double *mneq, const double *fneq,
                     double tau_prev, double *tau_out, double *S, double *tau_next) {
    double tau0 = 1.0 / p->s[L->nu_idx[0]];
    double c3 = 3.0 * p->smag_cs * p->smag_cs;
    *tau_next = tau0;
    if (p->closure == CL_SMAG_LAGGED) {
        strain_at(p, L, mneq, fneq, 1.0 / tau_prev, S);
        *tau_out = tau_prev;
        *tau_next = tau0 + c3 * strain_norm(L->q, S);
        return 0;
    }
    if (p->closure == CL_SMAG_DEV) {
        /* fixed point tau = tau0 + 3 Cs^2 |S_d(1/tau)| to a relative change of 1e-15 */
        double tau = tau0;
        int it;
        for (it = 1; it <= 200; ++it) {
            strain_at(p, L, mneq, fneq, 1.0 / tau, S);
            double tn = tau0 + c3 * dev_norm(L->q, S);
            double diff = fabs(tn - tau);
            tau = tn;
            if (diff <= 1e-15 * tn) break;
        }
        if (it > 200) it = 200;
        strain_at(p, L, mneq, fneq, 1.0 / tau, S);
        *tau_out = tau;
        *tau_next = tau;
        return it;
    }
    if (p->closure == CL_NEWTON) {
        /* rates used as given (the s_nu entries may differ from each other on the Chai route) */
        if (p->formula == F_YU)
            or_strain_yu(L->q, mneq, p->s, p->rho0, S);
        else
            or_strain_chai(L->q, fneq, p->s, p->rho0, S);
        *tau_out = tau0;
        return 0;
    }
    if (p->closure == CL_SMAG) {
        double tau = tau0;
        for (int k = 0; k < p->smag_iters; ++k) {
            strain_at(p, L, mneq, fneq, 1.0 / tau, S);
            tau = tau0 + 3.0 * p->smag_cs * p->smag_cs * strain_norm(L->q, S);
        }
        strain_at(p, L, mneq, fneq, 1.0 / tau, S);
        *tau_out = tau;
        *tau_next = tau;
        return p->smag_iters;
    }
    /* power law: nu = K |S|^(n-1), tau = 1/2 + 3 nu, clamped to [tau_min, tau_max] */
    double tau = tau0;
    int it = 0;
    for (it = 1; it <= p->pl_max_iter; ++it) {
        strain_at(p, L, mneq, fneq, 1.0 / tau, S);
        double g = strain_norm(L->q, S);
        double tn = 0.5 + 3.0 * p->pl_k * pow(g, p->pl_n - 1.0);
        if (!(tn >= p->pl_tau_min)) tn = p->pl_tau_min; /* also catches NaN */
        if (tn > p->pl_tau_max) tn = p->pl_tau_max;
        double diff = fabs(tn - tau);
        tau = tn;
        if (diff <= p->pl_tol * tn) break;
    }
    if (it > p->pl_max_iter) it = p->pl_max_iter;
    strain_at(p, L, mneq, fneq, 1.0 / tau, S);
    *tau_out = tau;
    *tau_next = tau;
    return it;
}

/* One collision at one node (eq. (mrteqvT) with the force source):
 *   fin: pre-collision populations (already pulled), F: force density at the node (d comps),
 *   tau_prev: the node's stored tau (lagged closure only; ignored otherwise).
 *   fout: post-collision populations; S: strain rate (n_strain comps) of the pre-collision state
 *   with the converged closure; tau: the effective tau; iters: closure sweeps; tau_next: the tau
 *   to store for the next step (may be NULL). */
int or_collide(const or_params *p, const double *fin, const double *F, double tau_prev, double *fout,
               double *S, double *tau_out, int *iters_out, double *tau_next) {
    const lattice_t *L = lattice(p->q);
    if (!L) return OR_ERR_ARG;
    const int q = L->q;
    double Fv[3] = {F ? F[0] : 0.0, F ? F[1] : 0.0, (F && L->d == 3) ? F[2] : 0.0};

    /* macroscopic: drho = sum f, j = sum c f + F/2 */
    double drho = 0.0, j[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < q; ++i) {
        drho += fin[i];
        for (int a = 0; a < 3; ++a) j[a] += L->c[i][a] * fin[i];
    }
    for (int a = 0; a < 3; ++a) j[a] += 0.5 * Fv[a];

    /* m = T f (dense) */
    double m[19], meq[19], feq[19], Fbar[19], TF[19];
    for (int k = 0; k < q; ++k) {
        double acc = 0.0;
        for (int i = 0; i < q; ++i) acc += L->T[k][i] * fin[i];
        m[k] = acc;
    }
    or_meq(q, drho, j, p->rho0, meq);
    or_feq(q, drho, j, p->rho0, feq);
    or_force_bar(q, j, p->rho0, Fv, Fbar);
    for (int k = 0; k < q; ++k) {
        double acc = 0.0;
        for (int i = 0; i < q; ++i) acc += L->T[k][i] * Fbar[i];
        TF[k] = acc;
    }

    /* effective non-equilibrium parts (force half-shift) */
    double mneq[19], fneq[19];
    for (int k = 0; k < q; ++k) mneq[k] = m[k] - meq[k] + 0.5 * TF[k];
    for (int i = 0; i < q; ++i) fneq[i] = fin[i] - feq[i] + 0.5 * Fbar[i];

    double Sl[6] = {0, 0, 0, 0, 0, 0}, tau = 0.0, tnext = 0.0;
    int iters = solve_tau(p, L, mneq, fneq, tau_prev, &tau, Sl, &tnext);

    /* rates of this collision */
    double s[19];
    for (int k = 0; k < q; ++k) s[k] = p->s[k];
    if (p->closure != CL_NEWTON)
        for (int k = 0; k < L->n_nu; ++k) s[L->nu_idx[k]] = 1.0 / tau;

    /* m* = m - L (m - m_eq) + (I - L/2) T Fbar ;  f* = T^-1 m* */
    double mstar[19];
    for (int k = 0; k < q; ++k) mstar[k] = m[k] - s[k] * (m[k] - meq[k]) + (1.0 - 0.5 * s[k]) * TF[k];
    for (int i = 0; i < q; ++i) {
        double acc = 0.0;
        for (int k = 0; k < q; ++k) acc += L->Tinv[i][k] * mstar[k];
        fout[i] = acc;
    }
    if (S)
        for (int c = 0; c < strain_components(q); ++c) S[c] = Sl[c];
    if (tau_out) *tau_out = tau;
    if (iters_out) *iters_out = iters;
    if (tau_next) *tau_next = tnext;
    return OR_OK;
}

/* ------------------------------------------------------------------------------------------ */
/* Grid: pull streaming with boundaries, whole steps, read-outs, initialisation                */
/* ------------------------------------------------------------------------------------------ */

static int check_grid(const or_params *p, int nx, int ny, int nz) {
    const lattice_t *L = lattice(p->q);
    if (!L || nx < 1 || ny < 1 || nz < 1) return OR_ERR_ARG;
    if (L->d == 2 && nz != 1) return OR_ERR_ARG;
    for (int a = 0; a < 3; ++a) {
        int per0 = p->bc[2 * a] == BC_PERIODIC, per1 = p->bc[2 * a + 1] == BC_PERIODIC;
        if (L->d == 2 && a == 2) continue;
        if (per0 != per1) return OR_ERR_ARG;
    }
    return OR_OK;
}

static long idx3(int nx, int ny, int x, int y, int z) { return ((long)z * ny + y) * nx + x; }

/* Pre-collision population i at node (x,y,z), pulled from the post-collision buffer fpost:
 * f_i(x) = f*_i(x - c_i) inside the domain (periodic faces wrap).  When x - c_i lies behind a
 * wall face, halfway bounce-back gives f_i(x) = f*_opp(i)(x); if it lies behind exactly one face
 * and that face moves with velocity u_w, the Ladd term 2 w_i rho0 (c_i . u_w) / cs2 is added. */
static double pull(const or_params *p, const lattice_t *L, const double *fpost, long N, int nx, int ny,
                   int nz, int x, int y, int z, int i) {
    int src[3] = {x - L->c[i][0], y - L->c[i][1], z - L->c[i][2]};
    int dims[3] = {nx, ny, nz};
    int outside = 0, face = -1;
    for (int a = 0; a < 3; ++a) {
        if (src[a] >= 0 && src[a] < dims[a]) continue;
        int f = 2 * a + (src[a] < 0 ? 0 : 1);
        if (L->d == 2 && a == 2) {
            src[a] = (src[a] % dims[a] + dims[a]) % dims[a];
            continue;
        }
        if (p->bc[f] == BC_PERIODIC) {
            src[a] = (src[a] % dims[a] + dims[a]) % dims[a];
        } else {
            outside++;
            face = f;
        }
    }
    if (outside == 0) return fpost[(long)i * N + idx3(nx, ny, src[0], src[1], src[2])];
    double v = fpost[(long)L->opp[i] * N + idx3(nx, ny, x, y, z)];
    if (outside == 1 && p->bc[face] == BC_LID) {
        double cu = 0.0;
        for (int a = 0; a < 3; ++a) cu += L->c[i][a] * p->lid_u[face][a];
        v += 2.0 * L->w[i] * p->rho0 * cu / CS2;
    }
    return v;
}

/* Collide one node of the grid from the post-collision buffer fpost (pull), without writing
 * the grid: used for whole steps and for sampled comparisons at large sizes.
 * force: NULL (none), or d values (uniform) when force_field == 0, or a d x N field.
 * tau_field: the stored tau of every node (N values; read by the lagged closure, which requires
 * it); tau_next: the node's tau for the next step (may be NULL). */
int or_node(const or_params *p, int nx, int ny, int nz, const double *fpost, const double *force,
            int force_field, const double *tau_field, int x, int y, int z, double *fout, double *S,
            double *tau, int *iters, double *fin_out, double *tau_next) {
    if (check_grid(p, nx, ny, nz) != OR_OK) return OR_ERR_ARG;
    const lattice_t *L = lattice(p->q);
    long N = (long)nx * ny * nz;
    double fin[19], F[3] = {0, 0, 0};
    for (int i = 0; i < L->q; ++i) fin[i] = pull(p, L, fpost, N, nx, ny, nz, x, y, z, i);
    if (force) {
        long n = idx3(nx, ny, x, y, z);
        for (int a = 0; a < L->d; ++a) F[a] = force_field ? force[(long)a * N + n] : force[a];
    }
    if (fin_out)
        for (int i = 0; i < L->q; ++i) fin_out[i] = fin[i];
    if (p->closure == CL_SMAG_LAGGED && !tau_field) return OR_ERR_ARG;
    double tp = tau_field ? tau_field[idx3(nx, ny, x, y, z)] : 0.0;
    return or_collide(p, fin, F, tp, fout, S, tau, iters, tau_next);
}

/* One full time step: fnew = collide(pull(fpost)).  Optional outputs of the pre-collision state
 * of this step: S (n_strain x N), tau (N), macroscopic drho (N) and u (d x N).
 * tau_field (N, lagged closure): the stored tau per node; tau_next (N, optional): the taus the
 * next step reads (may alias tau_field: each node reads only its own entry before writing it). */
int or_step(const or_params *p, int nx, int ny, int nz, const double *fpost, const double *force,
            int force_field, const double *tau_field, double *fnew, double *S, double *tau, double *drho,
            double *u, double *tau_next) {
    if (check_grid(p, nx, ny, nz) != OR_OK) return OR_ERR_ARG;
    const lattice_t *L = lattice(p->q);
    long N = (long)nx * ny * nz;
    int ns = n_strain(L->q);
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                long n = idx3(nx, ny, x, y, z);
                double fout[19], Sl[6], t, fin[19], tn;
                int it;
                int rc = or_node(p, nx, ny, nz, fpost, force, force_field, tau_field, x, y, z, fout, Sl, &t, &it,
                                 fin, &tn);
                if (rc != OR_OK) return rc;
                if (tau_next) tau_next[n] = tn;
                for (int i = 0; i < L->q; ++i) fnew[(long)i * N + n] = fout[i];
                if (S)
                    for (int c = 0; c < ns; ++c) S[(long)c * N + n] = Sl[c];
                if (tau) tau[n] = t;
                if (drho || u) {
                    double r = 0.0, j[3] = {0, 0, 0};
                    for (int i = 0; i < L->q; ++i) {
                        r += fin[i];
                        for (int a = 0; a < 3; ++a) j[a] += L->c[i][a] * fin[i];
                    }
                    if (drho) drho[n] = r;
                    if (u)
                        for (int a = 0; a < L->d; ++a) {
                            double Fa = force ? (force_field ? force[(long)a * N + n] : force[a]) : 0.0;
                            u[(long)a * N + n] = (j[a] + 0.5 * Fa) / p->rho0;
                        }
                }
            }
    return OR_OK;
}

/* tau that the closure assigns to a given strain rate S (not formed from populations) */
static double closure_tau_at(const or_params *p, const lattice_t *L, const double *S) {
    double tau0 = 1.0 / p->s[L->nu_idx[0]];
    double c3 = 3.0 * p->smag_cs * p->smag_cs;
    switch (p->closure) {
        case CL_SMAG:
        case CL_SMAG_LAGGED: return tau0 + c3 * strain_norm(L->q, S);
        case CL_SMAG_DEV: return tau0 + c3 * dev_norm(L->q, S);
        case CL_POWERLAW: {
            double tau = 0.5 + 3.0 * p->pl_k * pow(strain_norm(L->q, S), p->pl_n - 1.0);
            if (!(tau >= p->pl_tau_min)) tau = p->pl_tau_min;
            if (tau > p->pl_tau_max) tau = p->pl_tau_max;
            return tau;
        }
        default: return tau0;
    }
}

/* Initial state from macroscopic fields (Sec. 4.1, eq. (YuLuobasis)):
 *   pre-collision f(x, 0) = f_eq(drho, rho0 u) + T^-1 m_neq(grad u) - Fbar/2,
 * where m_neq holds only the first-order viscous moments.  D3Q19:
 *   m1 = -38/(3 s1) div j,  m9 = -2/(3 s_nu)(3 d_x j_x - div j),  m11 = -2/(3 s_nu)(d_y j_y - d_z j_z),
 *   m13 = -(d_x j_y + d_y j_x)/(3 s_nu),  m14 = -(d_y j_z + d_z j_y)/(3 s_nu),
 *   m15 = -(d_z j_x + d_x j_z)/(3 s_nu);
 * D2Q9 (same procedure with the D2Q9 Yu-type formula):
 *   m_e = -2 div j / s_e,  m_pxx = -2 (d_x j_x - d_y j_y)/(3 s_nu),  m_pxy = -(d_x j_y + d_y j_x)/(3 s_nu).
 * D3Q15 (the first-order Chapman-Enskog moments -(1/s_k) T (d_t + c.grad) f_eq worked out for the
 * d'Humieres basis):
 *   m_e = -2 div j / (3 s_e),  m_3pxx = -2 (3 d_x j_x - div j)/(3 s_nu),  m_pww = -2 (d_y j_y - d_z j_z)/(3 s_nu),
 *   m_pxy = -(d_x j_y + d_y j_x)/(3 s_nu),  m_pyz = -(d_y j_z + d_z j_y)/(3 s_nu),  m_pxz = -(d_x j_z + d_z j_x)/(3 s_nu).
 * s_nu is the closure's value for the given gradient (explicit, since S is given).
 * grad_u: d*d x N, entry (a*d + b) = d u_a / d x_b; NULL for a pure equilibrium.
 * The buffer written is the post-collision state of step -1: f(x,0) is un-streamed so that the
 * next pull returns exactly f(x,0).  tau_field (N, may be NULL) receives each node's closure tau
 * at the prescribed gradient (the lagged closure's first stored tau). */
int or_init(const or_params *p, int nx, int ny, int nz, const double *drho, const double *u,
            const double *grad_u, const double *force, int force_field, double *fpost, double *tau_field) {
    if (check_grid(p, nx, ny, nz) != OR_OK) return OR_ERR_ARG;
    const lattice_t *L = lattice(p->q);
    const int q = L->q, d = L->d;
    long N = (long)nx * ny * nz;
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                long n = idx3(nx, ny, x, y, z);
                double j[3] = {0, 0, 0}, F[3] = {0, 0, 0};
                for (int a = 0; a < d; ++a) j[a] = p->rho0 * u[(long)a * N + n];
                if (force)
                    for (int a = 0; a < d; ++a) F[a] = force_field ? force[(long)a * N + n] : force[a];
                double feq[19], Fbar[19], mneq[19];
                or_feq(q, drho[n], j, p->rho0, feq);
                or_force_bar(q, j, p->rho0, F, Fbar);
                for (int k = 0; k < q; ++k) mneq[k] = 0.0;
                double G[3][3] = {{0}}, Sx[6] = {0, 0, 0, 0, 0, 0};
                if (grad_u) {
                    for (int a = 0; a < d; ++a)
                        for (int b = 0; b < d; ++b) G[a][b] = p->rho0 * grad_u[(long)(a * d + b) * N + n];
                    if (d == 3) {
                        Sx[0] = G[0][0] / p->rho0;
                        Sx[1] = G[1][1] / p->rho0;
                        Sx[2] = G[2][2] / p->rho0;
                        Sx[3] = 0.5 * (G[0][1] + G[1][0]) / p->rho0;
                        Sx[4] = 0.5 * (G[1][2] + G[2][1]) / p->rho0;
                        Sx[5] = 0.5 * (G[0][2] + G[2][0]) / p->rho0;
                    } else {
                        Sx[0] = G[0][0] / p->rho0;
                        Sx[1] = G[1][1] / p->rho0;
                        Sx[2] = 0.5 * (G[0][1] + G[1][0]) / p->rho0;
                    }
                }
                /* the closure's tau at the prescribed strain rate (explicit, since S is given) */
                double tau_i = closure_tau_at(p, L, Sx);
                if (tau_field) tau_field[n] = tau_i;
                if (grad_u) {
                    double snu = p->closure == CL_NEWTON ? p->s[L->nu_idx[0]] : 1.0 / tau_i;
                    double divj = 0.0;
                    for (int a = 0; a < d; ++a) divj += G[a][a];
                    if (q == 19) {
                        mneq[1] = -38.0 / (3.0 * p->s[1]) * divj;
                        mneq[9] = -2.0 / (3.0 * snu) * (3.0 * G[0][0] - divj);
                        mneq[11] = -2.0 / (3.0 * snu) * (G[1][1] - G[2][2]);
                        mneq[13] = -(G[1][0] + G[0][1]) / (3.0 * snu);
                        mneq[14] = -(G[2][1] + G[1][2]) / (3.0 * snu);
                        mneq[15] = -(G[0][2] + G[2][0]) / (3.0 * snu);
                    } else if (q == 15) {
                        mneq[1] = -2.0 / (3.0 * p->s[1]) * divj;
                        mneq[9] = -2.0 / (3.0 * snu) * (3.0 * G[0][0] - divj);
                        mneq[10] = -2.0 / (3.0 * snu) * (G[1][1] - G[2][2]);
                        mneq[11] = -(G[1][0] + G[0][1]) / (3.0 * snu);
                        mneq[12] = -(G[2][1] + G[1][2]) / (3.0 * snu);
                        mneq[13] = -(G[0][2] + G[2][0]) / (3.0 * snu);
                    } else {
                        mneq[1] = -2.0 * divj / p->s[1];
                        mneq[7] = -2.0 * (G[0][0] - G[1][1]) / (3.0 * snu);
                        mneq[8] = -(G[1][0] + G[0][1]) / (3.0 * snu);
                    }
                }
                double f0[19];
                for (int i = 0; i < q; ++i) {
                    double acc = 0.0;
                    for (int k = 0; k < q; ++k) acc += L->Tinv[i][k] * mneq[k];
                    f0[i] = feq[i] + acc - 0.5 * Fbar[i];
                }
                /* un-stream: the entry that the pull of (x, i) reads receives f0[i] */
                for (int i = 0; i < q; ++i) {
                    int src[3] = {x - L->c[i][0], y - L->c[i][1], z - L->c[i][2]};
                    int dims[3] = {nx, ny, nz};
                    int outside = 0, face = -1;
                    for (int a = 0; a < 3; ++a) {
                        if (src[a] >= 0 && src[a] < dims[a]) continue;
                        int f = 2 * a + (src[a] < 0 ? 0 : 1);
                        if ((L->d == 2 && a == 2) || p->bc[f] == BC_PERIODIC) {
                            src[a] = (src[a] % dims[a] + dims[a]) % dims[a];
                        } else {
                            outside++;
                            face = f;
                        }
                    }
                    if (outside == 0) {
                        fpost[(long)i * N + idx3(nx, ny, src[0], src[1], src[2])] = f0[i];
                    } else {
                        double v = f0[i];
                        if (outside == 1 && p->bc[face] == BC_LID) {
                            double cu = 0.0;
                            for (int a = 0; a < 3; ++a) cu += L->c[i][a] * p->lid_u[face][a];
                            v -= 2.0 * L->w[i] * p->rho0 * cu / CS2;
                        }
                        fpost[(long)L->opp[i] * N + n] = v;
                    }
                }
            }
    return OR_OK;
}

/* Read-outs of the pre-collision state of the next step (pull from fpost):
 * strain rate by either formula with the converged closure, and macroscopic fields. */
int or_readout(const or_params *p, int nx, int ny, int nz, const double *fpost, const double *force,
               int force_field, const double *tau_field, double *S, double *tau, double *drho, double *u) {
    if (check_grid(p, nx, ny, nz) != OR_OK) return OR_ERR_ARG;
    long N = (long)nx * ny * nz;
    int q = p->q;
    double *scratch = (double *)malloc(sizeof(double) * (size_t)q * (size_t)N);
    if (!scratch) return OR_ERR_ARG;
    int rc = or_step(p, nx, ny, nz, fpost, force, force_field, tau_field, scratch, S, tau, drho, u, NULL);
    free(scratch);
    return rc;
}

/* Global sums of the pre-collision state: out = [sum f, sum j_x, sum j_y, (sum j_z)] with
 * j = sum c f + F/2, accumulated in plain FP64. */
int or_sums(const or_params *p, int nx, int ny, int nz, const double *fpost, const double *force,
            int force_field, double *out) {
    if (check_grid(p, nx, ny, nz) != OR_OK) return OR_ERR_ARG;
    const lattice_t *L = lattice(p->q);
    long N = (long)nx * ny * nz;
    for (int a = 0; a <= L->d; ++a) out[a] = 0.0;
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                long n = idx3(nx, ny, x, y, z);
                for (int i = 0; i < L->q; ++i) {
                    double f = pull(p, L, fpost, N, nx, ny, nz, x, y, z, i);
                    out[0] += f;
                    for (int a = 0; a < L->d; ++a) out[1 + a] += L->c[i][a] * f;
                }
                if (force)
                    for (int a = 0; a < L->d; ++a)
                        out[1 + a] += 0.5 * (force_field ? force[(long)a * N + n] : force[a]);
            }
    return OR_OK;
}
