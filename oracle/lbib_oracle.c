/*
 * lbib_oracle.c -- plain, slow, FP64 CPU oracle of the LB-IB time step.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls, links or
 * loads this file: only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header, table or helper with the CUDA
 * path (the CUDA path lives in paper_1907_00080_gb300/csrc and include/).
 *
 * What it computes (one time step n -> n+1, state (f^n, X^n, X^{n-1}, B^n, n)),
 * in the order below, each step following the paper passage it cites
 * (Coclite, "Vascular journey and adhesion mechanics of micro-sized carriers in
 * narrow capillaries", arXiv 1907.00080):
 *
 *   1. bond spring forces at X^n                       Eq. adhFor (Sec. 2.2)
 *   2. inter-membrane repulsion                        Eq. repFor (Sec. 2.2)
 *   3. stretching                                      Eq. strainFor
 *   4. bending                                         Eq. bendFor
 *   5. enclosed-area penalty                           Eq. areaFor
 *   6. IB weights: 3x3 nearest-node stencil, MLS with  Sec. 2.2 (MLS of Vanella
 *      a linear basis and Roma 3-point weights            et al.), Sec. 2.3
 *   7. spreading G = G_body + sum_v phi_v F_v          Sec. 2.2, Eq. ForcingTerm
 *   8. BGK collide with Guo forcing, pull streaming,   Eqs. BGK, feq,
 *      half-way bounce-back walls, periodic x            GaussHermite, forcedBGK,
 *                                                        ForcingTerm; Sec. 3
 *   9. interpolation U_v = sum_j phi_v(x_j) u(x_j)     Sec. 2.3 (blood cells)
 *  10. kinematic marker advance (BDF2)                 Eq. kinematicPos
 *      or, for dynamic particles, Newton's law under    Sec. 2.4: Eqs. hydroForP,
 *      internal and hydrodynamic forces, with the         hydroForNu, newtonSoft,
 *      fluid driven toward the particle velocity          verletPos, verletVel,
 *                                                         linearVelRig, angularVelRig
 *  11. bond rupture then formation at X^{n+1}          Sec. 2.2 (wall-particle)
 *  12. diagnostics (mass, enclosed area)               Sec. 2.1, Eq. areaFor
 *
 * The end of the file holds the forward-mode tangent of steps 1-10 in dual
 * numbers (orc_tangent_*), differentiated line by line from the code above,
 * with bond events (step 11) held at the primal's.
 *
 * Readings of passages the paper leaves open:
 *  - Eq. ForcingTerm is read as the standard Guo term
 *      F_i = (1 - 1/(2 tau)) w_i [3 (e_i - u) + 9 (e_i.u) e_i] . G
 *    and the momentum as rho u = sum_i f_i e_i + G/2 (Sec. 2.2, the "f_lb" in
 *    the text being the same body force).
 *  - walls are half-way bounce-back at y = -1/2 and y = NY - 1/2; or (walls =
 *    2) Zou and He's known-velocity condition on the wall rows y = 0 and
 *    y = NY - 1, with the populations' momentum the wall velocity less the
 *    Guo half-force of the node.
 *  - the MLS weight is the Roma 3-point kernel on the nine nearest nodes; where
 *    all nine nodes are fluid the MLS shape function equals the Roma weight
 *    exactly and is taken as such; near walls the out-of-fluid nodes are dropped
 *    and the 3x3 MLS system is solved.
 *  - bending: theta is the signed turning angle, n_v the normalised sum of the
 *    two adjacent outward edge normals; the left neighbour gets l_L/(l_L+l_R).
 *  - area: shoelace on the vertices, p_ref = 1/3, force split 1/2 + 1/2.
 *  - repulsion acts for d < d_rep, along the vertex's own inward normal.
 *  - bond force is along ligand->receptor; bond kinetics are Dembo-type forward
 *    and reverse probabilities (the paper defers their form to a citation).
 *  - first step advances with forward Euler (BDF2 needs two past positions).
 *  - dynamic particles: the fluid side of the coupling ("weak coupling",
 *    Sec. 2.4) is direct forcing, F^ib = 2 dV (u_particle - U~) spread with
 *    the IB shape functions; the stresses are evaluated on the flow at the
 *    start of the step; viscous stress rho_0 nu (grad u + grad u^T); vertex
 *    mass rho_P A_0 / n; rigid bodies turn about their area centroid; the
 *    particles start at rest.
 *  - random numbers: Philox4x64-10 (Salmon et al., SC'11), counter
 *    (step, ligand, receptor, tag), key (seed, instance); u = (x0 >> 11) 2^-53.
 *
 * Build:  gcc -O2 -std=c11 -ffp-contract=off -fPIC -shared lbib_oracle.c -lm
 * (no FMA contraction, so every product and sum is rounded as written).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef __FP_FAST_FMA
/* contraction is disabled on the command line; nothing here relies on it */
#endif

/* ------------------------------------------------------------------------- */
/* D2Q9 lattice, Eq. GaussHermite and the weights that follow it (Sec. 2.1).  */
/* i = 0: rest; i = 1..4: (cos((i-1)pi/2), sin((i-1)pi/2));                    */
/* i = 5..8: sqrt(2) (cos((2i-9)pi/4), sin((2i-9)pi/4)).                        */
/* ------------------------------------------------------------------------- */
static const int EX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double W9[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,
                             1.0 / 9.0,  1.0 / 9.0,  1.0 / 36.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

static int opposite(int i) {
    /* the direction with e_j = -e_i, found by search rather than a table */
    for (int j = 0; j < 9; ++j)
        if (EX[j] == -EX[i] && EY[j] == -EY[i]) return j;
    return -1;
}

static long imod(long a, long m) {
    long r = a % m;
    return r < 0 ? r + m : r;
}

/* ------------------------------------------------------------------------- */
/* Simulation state                                                           */
/* ------------------------------------------------------------------------- */
typedef struct {
    int nx, ny;
    double tau;
    double gx, gy;    /* uniform body force G_body (Sec. 3 drive)        */
    int walls;        /* 0: periodic in y too; 1: half-way bounce-back walls in y;
                         2: Zou-He known-velocity walls on the rows y = 0, NY - 1 */
    double *f;        /* f^n, [9][ny][nx], pre-collision                 */
    double *rho, *ux, *uy; /* moments of the last collide                */
    double *Gx, *Gy;  /* force field used by the last collide           */
    double *ftmp;

    /* membranes (closed rings, CCW) */
    int nmem, nv;
    int *mem_off, *mem_n, *mem_kind;
    double *mem_ks, *mem_kb, *mem_ka, *mem_A0;
    int *vert_mem;
    double *x, *y, *xp, *yp;   /* X^n and X^{n-1}, unwrapped */
    double *fx, *fy;           /* F^n                         */
    double *l0, *th0;          /* rest length of element v=(v,v+1); rest angle at v */
    double *wgt;               /* 9 weights per vertex, last step */
    long *widx;                /* 9 node indices per vertex      */
    double *Ux, *Uy;           /* interpolated velocity, last step */

    /* ligands (one per listed element) and receptors */
    int nlig;
    int *lig_elem;             /* global element id (= first vertex id) */
    int nrec;
    double *rx, *ry;
    int *bond_of_lig, *owner_of_rec;
    double d_cut, y_eq, sigma, kf_dt, kr0_dt, beta_f, beta_r, d_break;
    uint64_t seed, instance;

    double d_rep, p_ref;
    double uw_bot, uw_top;     /* x velocities of the lower and upper walls */
    long step;

    /* dynamic particles (kinds 2 and 3, Sec. 2.4) */
    double *mem_rhop;          /* particle density over fluid density        */
    double *mem_J0;            /* polar second moment of area of the rest shape about its centroid */
    double *mem_rb;            /* rigid state per membrane: u, v, u_prev, v_prev, omega, omega_prev */
    double *vx, *vy;           /* particle velocity of each vertex, u_v^n    */
    double *hx, *hy;           /* hydrodynamic force on each vertex, last step */
    double *ibx, *iby;         /* force spread into the fluid for each dynamic vertex, last step */
} orc_sim;

/* ------------------------------------------------------------------------- */
/* Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11), written from its        */
/* published definition: ten rounds of two 64x64->128 multiplies, a key       */
/* schedule bumped by the Weyl constants between rounds.                      */
/* ------------------------------------------------------------------------- */
void orc_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t K0 = 0x9E3779B97F4A7C15ULL, K1 = 0xBB67AE8584CAA73BULL;
    uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += K0; k1 += K1; }
        unsigned __int128 p0 = (unsigned __int128)M0 * x0;
        unsigned __int128 p1 = (unsigned __int128)M1 * x2;
        uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
        uint64_t n0 = hi1 ^ x1 ^ k0;
        uint64_t n1 = lo1;
        uint64_t n2 = hi0 ^ x3 ^ k1;
        uint64_t n3 = lo0;
        x0 = n0; x1 = n1; x2 = n2; x3 = n3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* uniform draw in [0,1) for bond decision `tag` (0 = formation, 1 = rupture) */
double orc_uniform(uint64_t seed, uint64_t instance, long step, long lig, long rec, long tag) {
    uint64_t c[4] = {(uint64_t)step, (uint64_t)lig, (uint64_t)rec, (uint64_t)tag};
    uint64_t k[2] = {seed, instance};
    uint64_t o[4];
    orc_philox4x64_10(c, k, o);
    return (double)(o[0] >> 11) * (1.0 / 9007199254740992.0); /* 2^-53 */
}

/* ------------------------------------------------------------------------- */
/* LB pieces                                                                  */
/* ------------------------------------------------------------------------- */

/* Eq. feq with c_s^2 = 1/3: w_i rho [1 + 3 e.u + 9/2 (e.u)^2 - 3/2 u.u] */
void orc_equilibrium(double rho, double ux, double uy, double feq[9]) {
    double uu = ux * ux + uy * uy;
    for (int i = 0; i < 9; ++i) {
        double eu = EX[i] * ux + EY[i] * uy;
        feq[i] = W9[i] * rho * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu);
    }
}

/* Eq. ForcingTerm (Guo): (1 - 1/(2 tau)) w_i [(e_i - u)/c_s^2 + (e_i.u) e_i / c_s^4] . G */
void orc_guo_source(double tau, double ux, double uy, double gx, double gy, double F[9]) {
    double pre = 1.0 - 1.0 / (2.0 * tau);
    for (int i = 0; i < 9; ++i) {
        double eu = EX[i] * ux + EY[i] * uy;
        double cx = 3.0 * (EX[i] - ux) + 9.0 * eu * EX[i];
        double cy = 3.0 * (EY[i] - uy) + 9.0 * eu * EY[i];
        F[i] = pre * W9[i] * (cx * gx + cy * gy);
    }
}

/* moments with the Guo half-force correction (Sec. 2.1, Sec. 2.2):
 * rho = sum f_i ; rho u = sum f_i e_i + G/2 */
static void moments_at(const double *f, long N, long node, double gx, double gy,
                       double *rho, double *ux, double *uy) {
    double r = 0.0, jx = 0.0, jy = 0.0;
    for (int i = 0; i < 9; ++i) {
        double fi = f[i * N + node];
        r += fi;
        jx += fi * EX[i];
        jy += fi * EY[i];
    }
    jx += 0.5 * gx;
    jy += 0.5 * gy;
    *rho = r;
    *ux = jx / r;
    *uy = jy / r;
}

/* streaming of a post-collision field fstar into fout (Eq. BGK left-hand side):
 * f_i(x, t+1) = f*_i(x - e_i); periodic in x; in y periodic (walls = 0) or
 * half-way bounce-back f_i(x, t+1) = f*_opp(i)(x) when x - e_i is a wall.  A
 * wall moving along x with velocity u_w (the Couette set-up of Sec. 4) adds the
 * momentum it imparts, 2 w_i rho_w (e_i . u_w) / c_s^2 with rho_w = 1 (the
 * bounce-back rule for moving walls of Ladd, J. Fluid Mech. 271, 1994). */
/* Zou and He's known-velocity condition (Sec. 2.1; Zou & He, Phys. Fluids 9,
 * 1997) on a wall row (wet nodes: y = 0 is the lower wall, y = NY - 1 the
 * upper one).  After streaming, the three populations that would come from
 * outside the fluid are unknown: at the lower wall f_2, f_5, f_6, at the upper
 * f_4, f_7, f_8.  With the wall's velocity (u_w, 0) and the known populations,
 * density and momentum fix them: rho = f_0 + f_1 + f_3 + 2 (the three known
 * populations leaving toward the wall's outside) + j_y (j_y signed toward the
 * inside), and the unknown normal population is its opposite plus 2/3 j_y,
 * the two unknown diagonals their opposites -+ (f_1 - f_3)/2 +- j_x/2 + j_y/6.
 * The momentum the populations carry is the known velocity less the Guo
 * half-force of the node (rho u = sum f e + G/2, Sec. 2.2):
 * j = rho (u_w, 0) - G/2, so that the collision sees u = (u_w, 0). */
static void zou_he_node(const orc_sim *s, double *f, long N, long node, int lower, double gx, double gy) {
    double uw = lower ? s->uw_bot : s->uw_top;
    double f0 = f[0 * N + node], f1 = f[1 * N + node], f3 = f[3 * N + node];
    if (lower) {
        double f4 = f[4 * N + node], f7 = f[7 * N + node], f8 = f[8 * N + node];
        double jy = -0.5 * gy;                      /* toward the inside: +y */
        double rho = f0 + f1 + f3 + 2.0 * (f4 + f7 + f8) + jy;
        double jx = rho * uw - 0.5 * gx;
        f[2 * N + node] = f4 + (2.0 / 3.0) * jy;
        f[5 * N + node] = f7 - 0.5 * (f1 - f3) + 0.5 * jx + (1.0 / 6.0) * jy;
        f[6 * N + node] = f8 + 0.5 * (f1 - f3) - 0.5 * jx + (1.0 / 6.0) * jy;
    } else {
        double f2 = f[2 * N + node], f5 = f[5 * N + node], f6 = f[6 * N + node];
        double jy = -0.5 * gy;                      /* y momentum the populations carry */
        double rho = f0 + f1 + f3 + 2.0 * (f2 + f5 + f6) - jy;
        double jx = rho * uw - 0.5 * gx;
        f[4 * N + node] = f2 - (2.0 / 3.0) * jy;
        f[7 * N + node] = f5 + 0.5 * (f1 - f3) - 0.5 * jx - (1.0 / 6.0) * jy;
        f[8 * N + node] = f6 - 0.5 * (f1 - f3) + 0.5 * jx - (1.0 / 6.0) * jy;
    }
}

void orc_stream(const orc_sim *s, const double *fstar, double *fout) {
    long nx = s->nx, ny = s->ny, N = nx * ny;
    for (int i = 0; i < 9; ++i) {
        int o = opposite(i);
#pragma omp parallel for schedule(static)
        for (long y = 0; y < ny; ++y) {
            for (long x = 0; x < nx; ++x) {
                long sy = y - EY[i];
                long sx = imod(x - EX[i], nx);
                double v;
                if (s->walls == 2 && (sy < 0 || sy >= ny)) {
                    v = 0.0;  /* unknown: Zou-He below */
                } else if (s->walls && (sy < 0 || sy >= ny)) {
                    double uw = sy < 0 ? s->uw_bot : s->uw_top;
                    v = fstar[o * N + y * nx + x] + 6.0 * W9[i] * (EX[i] * uw);
                } else {
                    sy = imod(sy, ny);
                    v = fstar[i * N + sy * nx + sx];
                }
                fout[i * N + y * nx + x] = v;
            }
        }
    }
    /* Zou-He walls: the unknown populations of the wall rows as the known
     * velocity fixes them; the collision redoes this with the node's force */
    if (s->walls == 2) {
        for (long x = 0; x < nx; ++x) {
            zou_he_node(s, fout, N, x, 1, 0.0, 0.0);
            zou_he_node(s, fout, N, (ny - 1) * nx + x, 0, 0.0, 0.0);
        }
    }
}

void orc_moments(const orc_sim *s, const double *f, const double *Gx, const double *Gy,
                 double *rho, double *ux, double *uy) {
    long N = (long)s->nx * s->ny;
    for (long n = 0; n < N; ++n)
        moments_at(f, N, n, Gx ? Gx[n] : s->gx, Gy ? Gy[n] : s->gy, &rho[n], &ux[n], &uy[n]);
}

/* Eq. forcedBGK with Delta t = 1, then streaming; stores rho, u */
static void collide_and_stream(orc_sim *s) {
    long N = (long)s->nx * s->ny;
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
        double feq[9], F[9];
        double rho, ux, uy;
        double gx = s->Gx[n], gy = s->Gy[n];
        if (s->walls == 2 && (n < s->nx || n >= N - s->nx))
            zou_he_node(s, s->f, N, n, n < s->nx, gx, gy);
        moments_at(s->f, N, n, gx, gy, &rho, &ux, &uy);
        s->rho[n] = rho; s->ux[n] = ux; s->uy[n] = uy;
        orc_equilibrium(rho, ux, uy, feq);
        orc_guo_source(s->tau, ux, uy, gx, gy, F);
        for (int i = 0; i < 9; ++i) {
            double fi = s->f[i * N + n];
            s->ftmp[i * N + n] = fi - (fi - feq[i]) / s->tau + F[i];
        }
    }
    orc_stream(s, s->ftmp, s->f);
}

/* ------------------------------------------------------------------------- */
/* Immersed boundary: Roma kernel, MLS shape functions, interp and spread     */
/* ------------------------------------------------------------------------- */

/* Roma, Peskin & Berger (1999) three-point regularised delta */
double orc_roma(double r) {
    double a = fabs(r);
    if (a <= 0.5) return (1.0 + sqrt(1.0 - 3.0 * a * a)) / 3.0;
    if (a <= 1.5) {
        double b = 1.0 - a;
        return (5.0 - 3.0 * a - sqrt(1.0 - 3.0 * b * b)) / 6.0;
    }
    return 0.0;
}

/* Shape functions of one Lagrangian point (Sec. 2.2 MLS exchange; Sec. 2.3
 * nine Eulerian points).  Nodes are (i0+a, j0+b), a,b in {-1,0,1}, stored
 * row-major in b then a; idx receives the linear node index (-1 if dropped). */
void orc_ib_weights(const orc_sim *s, double px, double py, double w[9], long idx[9]) {
    long i0 = (long)floor(px + 0.5), j0 = (long)floor(py + 0.5);
    double Wr[9], rx[9], ry[9];
    int nvalid = 0;
    for (int b = -1; b <= 1; ++b) {
        for (int a = -1; a <= 1; ++a) {
            int k = (b + 1) * 3 + (a + 1);
            long i = i0 + a, j = j0 + b;
            rx[k] = (double)i - px;
            ry[k] = (double)j - py;
            int inside = s->walls ? (j >= 0 && j < s->ny) : 1;
            if (inside) {
                Wr[k] = orc_roma(rx[k]) * orc_roma(ry[k]);
                idx[k] = imod(j, s->ny) * s->nx + imod(i, s->nx);
                ++nvalid;
            } else {
                Wr[k] = 0.0;
                idx[k] = -1;
            }
        }
    }
    if (nvalid == 9) {
        /* full stencil: the MLS system is diag(1, ., .) and phi_j = W_j */
        for (int k = 0; k < 9; ++k) w[k] = Wr[k];
        return;
    }
    /* MLS with basis p = [1, rx, ry]: A = sum W p p^T, phi_j = W_j p_j^T A^{-1} e_1 */
    double A[3][3] = {{0}};
    double sumW = 0.0;
    for (int k = 0; k < 9; ++k) {
        double p[3] = {1.0, rx[k], ry[k]};
        sumW += Wr[k];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) A[r][c] += Wr[k] * p[r] * p[c];
    }
    /* first column of the inverse by cofactors: c = A^{-1} e_1 */
    double c00 = A[1][1] * A[2][2] - A[1][2] * A[2][1];
    double c10 = -(A[1][0] * A[2][2] - A[1][2] * A[2][0]);
    double c20 = A[1][0] * A[2][1] - A[1][1] * A[2][0];
    double det = A[0][0] * c00 + A[0][1] * c10 + A[0][2] * c20;
    if (det > 1e-10) {
        double cv[3] = {c00 / det, c10 / det, c20 / det};
        for (int k = 0; k < 9; ++k)
            w[k] = Wr[k] * (cv[0] + cv[1] * rx[k] + cv[2] * ry[k]);
    } else if (sumW > 0.0) {
        /* degenerate support (point outside the fluid): normalised weights */
        for (int k = 0; k < 9; ++k) w[k] = Wr[k] / sumW;
    } else {
        for (int k = 0; k < 9; ++k) w[k] = 0.0;
    }
}

/* interpolation of a node field (ux, uy) to points (Sec. 2.3) */
void orc_interp(const orc_sim *s, const double *ux, const double *uy, int np,
                const double *px, const double *py, double *Ux, double *Uy) {
    for (int v = 0; v < np; ++v) {
        double w[9];
        long idx[9];
        orc_ib_weights(s, px[v], py[v], w, idx);
        double a = 0.0, b = 0.0;
        for (int k = 0; k < 9; ++k) {
            if (idx[k] < 0) continue;
            a += w[k] * ux[idx[k]];
            b += w[k] * uy[idx[k]];
        }
        Ux[v] = a;
        Uy[v] = b;
    }
}

/* spreading of point forces with the same shape functions (adds into Gx, Gy) */
void orc_spread(const orc_sim *s, int np, const double *px, const double *py,
                const double *Fx, const double *Fy, double *Gx, double *Gy) {
    for (int v = 0; v < np; ++v) {
        double w[9];
        long idx[9];
        orc_ib_weights(s, px[v], py[v], w, idx);
        for (int k = 0; k < 9; ++k) {
            if (idx[k] < 0) continue;
            Gx[idx[k]] += w[k] * Fx[v];
            Gy[idx[k]] += w[k] * Fy[v];
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Membrane mechanics on one closed ring (vertex v joins v+1 mod n)           */
/* ------------------------------------------------------------------------- */

/* enclosed area by the shoelace formula, taken about vertex 0 (Eq. areaFor's
 * Green's-theorem area of the polygon) */
double orc_ring_area(int n, const double *x, const double *y) {
    double s = 0.0;
    double xr = x[0], yr = y[0];
    for (int v = 0; v < n; ++v) {
        int w = (v + 1) % n;
        s += (x[v] - xr) * (y[w] - yr) - (x[w] - xr) * (y[v] - yr);
    }
    return 0.5 * s;
}

/* signed turning angle at v and the vertex outward normal */
static void vertex_geometry(int n, const double *x, const double *y, int v,
                            double *theta, double *nvx, double *nvy,
                            double *lL, double *lR) {
    int L = (v + n - 1) % n, R = (v + 1) % n;
    double eLx = x[v] - x[L], eLy = y[v] - y[L];
    double eRx = x[R] - x[v], eRy = y[R] - y[v];
    double a = sqrt(eLx * eLx + eLy * eLy);
    double b = sqrt(eRx * eRx + eRy * eRy);
    double cr = eLx * eRy - eLy * eRx;
    double dt = eLx * eRx + eLy * eRy;
    *theta = atan2(cr, dt);
    /* outward edge normal of a CCW ring: (e_y, -e_x)/|e| */
    double nx_ = eLy / a + eRy / b;
    double ny_ = -eLx / a - eRx / b;
    double nn = sqrt(nx_ * nx_ + ny_ * ny_);
    *nvx = nx_ / nn;
    *nvy = ny_ / nn;
    *lL = a;
    *lR = b;
}

/* rest state: element lengths, vertex angles and area (stress-free shape) */
void orc_ring_rest(int n, const double *x, const double *y, double *l0, double *th0, double *A0) {
    for (int v = 0; v < n; ++v) {
        int w = (v + 1) % n;
        double dx = x[v] - x[w], dy = y[v] - y[w];
        l0[v] = sqrt(dx * dx + dy * dy);
        double th, a, b, c, d;
        vertex_geometry(n, x, y, v, &th, &a, &b, &c, &d);
        th0[v] = th;
    }
    *A0 = orc_ring_area(n, x, y);
}

/* internal forces of one ring; `which` bit 1 stretch, 2 bend, 4 area.
 * Adds into fx, fy. */
void orc_ring_forces(int n, const double *x, const double *y, const double *l0,
                     const double *th0, double A0, double ks, double kb, double ka,
                     double p_ref, int which, double *fx, double *fy) {
    if (which & 1) {
        /* Eq. strainFor: F_1 = -k_s (l - l_0) r_12 / l, F_2 = -k_s (l - l_0) r_21 / l */
        for (int v = 0; v < n; ++v) {
            int w = (v + 1) % n;
            double r12x = x[v] - x[w], r12y = y[v] - y[w];
            double l = sqrt(r12x * r12x + r12y * r12y);
            double c = -ks * (l - l0[v]) / l;
            fx[v] += c * r12x;
            fy[v] += c * r12y;
            fx[w] -= c * r12x;
            fy[w] -= c * r12y;
        }
    }
    if (which & 2) {
        /* Eq. bendFor */
        for (int v = 0; v < n; ++v) {
            int L = (v + n - 1) % n, R = (v + 1) % n;
            double th, nvx, nvy, lL, lR;
            vertex_geometry(n, x, y, v, &th, &nvx, &nvy, &lL, &lR);
            double m = kb * (th - th0[v]);
            double sL = lL / (lL + lR), sR = lR / (lL + lR);
            fx[L] += m * sL * nvx;
            fy[L] += m * sL * nvy;
            fx[v] -= m * nvx;
            fy[v] -= m * nvy;
            fx[R] += m * sR * nvx;
            fy[R] += m * sR * nvy;
        }
    }
    if (which & 4) {
        /* Eq. areaFor: F_l = -k_a (1 - A/A_0) p_ref n_l^- l_l, half to each end */
        double A = orc_ring_area(n, x, y);
        double c = -ka * (1.0 - A / A0) * p_ref;
        for (int v = 0; v < n; ++v) {
            int w = (v + 1) % n;
            double ex = x[w] - x[v], ey = y[w] - y[v];
            /* inward unit normal times the element length: (-e_y, e_x) */
            double Fx = c * (-ey), Fy = c * ex;
            fx[v] += 0.5 * Fx;
            fy[v] += 0.5 * Fy;
            fx[w] += 0.5 * Fx;
            fy[w] += 0.5 * Fy;
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Dynamic IB for particles (Sec. 2.4)                                        */
/*                                                                           */
/* Particles of kind 2 (deformable) and 3 (rigid) move by Newton's law        */
/* under their internal forces and the hydrodynamic stresses of Eqs.          */
/* hydroForP / hydroForNu, instead of with the fluid.  The fluid feels them   */
/* through a forcing term that drives its velocity at the vertices toward the */
/* particle's (the paper's "effective forcing term", read as direct forcing:  */
/* Uhlmann, J. Comput. Phys. 209, 2005; with the MLS transfer of Vanella &    */
/* Balaras, J. Comput. Phys. 228, 2009).                                      */
/* ------------------------------------------------------------------------- */

/* Area, area centroid and polar second moment about the centroid of a closed
 * CCW polygon, summed over the triangles (vertex 0, v, v+1): with a, b their
 * corners relative to vertex 0 and c = a x b, the triangle has area c/2,
 * centroid (a + b)/3 and polar moment c (|a|^2 + a.b + |b|^2) / 12 about
 * vertex 0; the parallel-axis theorem moves the sum to the centroid.  The
 * centroid is returned relative to vertex 0. */
void orc_ring_mass_properties(int n, const double *x, const double *y, double *A, double *cx,
                              double *cy, double *J) {
    double s2 = 0.0, sx = 0.0, sy = 0.0, sj = 0.0;
    for (int v = 0; v < n; ++v) {
        int w = (v + 1) % n;
        double ax = x[v] - x[0], ay = y[v] - y[0];
        double bx = x[w] - x[0], by = y[w] - y[0];
        double c = ax * by - ay * bx;
        s2 += c;
        sx += c * (ax + bx);
        sy += c * (ay + by);
        sj += c * ((ax * ax + ay * ay) + (ax * bx + ay * by) + (bx * bx + by * by));
    }
    double area = 0.5 * s2;
    double gx = sx / (3.0 * s2), gy = sy / (3.0 * s2);
    *A = area;
    *cx = gx;
    *cy = gy;
    *J = sj / 12.0 - area * (gx * gx + gy * gy);
}

/* MLS fit at a point q (Sec. 2.2: the moving-least-squares transfer; the
 * probe derivatives of Eqs. hydroForP / hydroForNu): over the 3x3 nodes
 * nearest to q that lie in the fluid, with Roma weights W_j and the linear
 * basis p_j = [1, x_j - q_x, y_j - q_y], A = sum_j W_j p_j p_j^T and a field g
 * is fitted by a = A^{-1} sum_j W_j p_j g_j: a_0 is its value at q, a_1 and
 * a_2 its x and y derivatives.  phi[r][k] = W_k (A^{-1} p_k)_r, so that
 * a_r = sum_k phi[r][k] g(idx[k]).  When A is singular (q too far outside the
 * fluid) the value falls back to the normalised weights and the gradient to
 * zero. */
void orc_mls_shape(const orc_sim *s, double qx, double qy, double phi[3][9], long idx[9]) {
    long i0 = (long)floor(qx + 0.5), j0 = (long)floor(qy + 0.5);
    double Wr[9], rx[9], ry[9];
    for (int b = -1; b <= 1; ++b) {
        for (int a = -1; a <= 1; ++a) {
            int k = (b + 1) * 3 + (a + 1);
            long i = i0 + a, j = j0 + b;
            rx[k] = (double)i - qx;
            ry[k] = (double)j - qy;
            int inside = s->walls ? (j >= 0 && j < s->ny) : 1;
            if (inside) {
                Wr[k] = orc_roma(rx[k]) * orc_roma(ry[k]);
                idx[k] = imod(j, s->ny) * s->nx + imod(i, s->nx);
            } else {
                Wr[k] = 0.0;
                idx[k] = -1;
            }
        }
    }
    double A[3][3] = {{0}};
    double sumW = 0.0;
    for (int k = 0; k < 9; ++k) {
        double p[3] = {1.0, rx[k], ry[k]};
        sumW += Wr[k];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) A[r][c] += Wr[k] * p[r] * p[c];
    }
    /* inverse by the adjugate (A is symmetric, so is its cofactor matrix) */
    double cof[3][3];
    cof[0][0] = A[1][1] * A[2][2] - A[1][2] * A[2][1];
    cof[0][1] = -(A[1][0] * A[2][2] - A[1][2] * A[2][0]);
    cof[0][2] = A[1][0] * A[2][1] - A[1][1] * A[2][0];
    cof[1][1] = A[0][0] * A[2][2] - A[0][2] * A[2][0];
    cof[1][2] = -(A[0][0] * A[2][1] - A[0][1] * A[2][0]);
    cof[2][2] = A[0][0] * A[1][1] - A[0][1] * A[1][0];
    cof[1][0] = cof[0][1];
    cof[2][0] = cof[0][2];
    cof[2][1] = cof[1][2];
    double det = A[0][0] * cof[0][0] + A[0][1] * cof[0][1] + A[0][2] * cof[0][2];
    for (int k = 0; k < 9; ++k) {
        if (det > 1e-10) {
            for (int r = 0; r < 3; ++r)
                phi[r][k] = Wr[k] * (cof[r][0] + cof[r][1] * rx[k] + cof[r][2] * ry[k]) / det;
        } else {
            phi[0][k] = sumW > 0.0 ? Wr[k] / sumW : 0.0;
            phi[1][k] = 0.0;
            phi[2][k] = 0.0;
        }
    }
}

/* value and gradient of a node field at q by the MLS fit */
void orc_mls_fit(const orc_sim *s, double qx, double qy, const double *g, double out[3]) {
    double phi[3][9];
    long idx[9];
    orc_mls_shape(s, qx, qy, phi, idx);
    for (int r = 0; r < 3; ++r) {
        double a = 0.0;
        for (int k = 0; k < 9; ++k)
            if (idx[k] >= 0) a += phi[r][k] * g[idx[k]];
        out[r] = a;
    }
}

/* the flow seen by the particles at the start of a step: rho and
 * u = (sum f e + G_body/2) / rho of the pre-collision populations f^n (the
 * IB forces of the step are not yet known), and the pressure relative to
 * the reference state, p = c_s^2 (rho - 1) with c_s^2 = 1/3 (Sec. 2.1) */
static void flow_at(const orc_sim *s, long node, double *p, double *ux, double *uy) {
    long N = (long)s->nx * s->ny;
    double rho;
    moments_at(s->f, N, node, s->gx, s->gy, &rho, ux, uy);
    *p = (rho - 1.0) / 3.0;
}

/* Eqs. hydroForP and hydroForNu on every element l = (v, v+1) of membrane m:
 * F_l = (-p n_l + tau . n_l) l_l with n_l the outward unit normal of the CCW
 * element, p and the velocity gradient taken from the MLS fit at the probe
 * point c_l + 1.2 n_l (c_l the element centroid), and the viscous stress
 * tau = rho_0 nu (grad u + grad u^T), rho_0 = 1, nu = (tau_LB - 1/2) / 3.
 * fe receives 2 n values (x, y per element). */
void orc_hydro_element_forces(const orc_sim *s, int m, double *fe) {
    int off = s->mem_off[m], n = s->mem_n[m];
    double nu = (s->tau - 0.5) / 3.0;
    for (int l = 0; l < n; ++l) {
        int v = off + l, w = off + (l + 1) % n;
        double ex = s->x[w] - s->x[v], ey = s->y[w] - s->y[v];
        double len = sqrt(ex * ex + ey * ey);
        double nx = ey / len, ny = -ex / len;
        double qx = 0.5 * (s->x[v] + s->x[w]) + 1.2 * nx;
        double qy = 0.5 * (s->y[v] + s->y[w]) + 1.2 * ny;
        double phi[3][9];
        long idx[9];
        orc_mls_shape(s, qx, qy, phi, idx);
        double p = 0.0, dux = 0.0, duy = 0.0, dvx = 0.0, dvy = 0.0;
        for (int k = 0; k < 9; ++k) {
            if (idx[k] < 0) continue;
            double pk, uk, vk;
            flow_at(s, idx[k], &pk, &uk, &vk);
            p += phi[0][k] * pk;
            dux += phi[1][k] * uk;
            duy += phi[2][k] * uk;
            dvx += phi[1][k] * vk;
            dvy += phi[2][k] * vk;
        }
        double txx = 2.0 * nu * dux, tyy = 2.0 * nu * dvy, txy = nu * (duy + dvx);
        fe[2 * l] = (-p * nx + (txx * nx + txy * ny)) * len;
        fe[2 * l + 1] = (-p * ny + (txy * nx + tyy * ny)) * len;
    }
}

static int is_dynamic(int kind) { return kind == 2 || kind == 3; }

/* For every dynamic membrane at X^n: the hydrodynamic force on each vertex
 * (half of each adjacent element's force, as the element forces of Eq. areaFor
 * are shared) is added to its total force F_v of Eq. newtonSoft, and the
 * force the vertex exerts on the fluid is
 *   F^ib_v = 2 dV_v (u_v - U~_v),
 * with u_v the particle velocity at the vertex, U~_v the interpolation of
 * the flow at the start of the step (same shape functions as the
 * kinematic markers), and dV_v = (l_L + l_R) / 2 the vertex's share of the
 * contour times Delta x = 1.  With Guo forcing a node's velocity carries half
 * the force it receives (rho u = sum f e + G/2, rho ~ 1): the factor 2 makes
 * F^ib the force that would bring the local velocity to u_v in one step. */
static void dynamic_coupling(orc_sim *s) {
    for (int m = 0; m < s->nmem; ++m) {
        if (!is_dynamic(s->mem_kind[m])) continue;
        int off = s->mem_off[m], n = s->mem_n[m];
        double *fe = (double *)malloc(sizeof(double) * 2 * (size_t)n);
        orc_hydro_element_forces(s, m, fe);
        for (int k = 0; k < n; ++k) {
            int v = off + k, L = off + (k + n - 1) % n, R = off + (k + 1) % n;
            int kl = (k + n - 1) % n;
            double hx = 0.5 * (fe[2 * kl] + fe[2 * k]);
            double hy = 0.5 * (fe[2 * kl + 1] + fe[2 * k + 1]);
            s->hx[v] = hx;
            s->hy[v] = hy;
            s->fx[v] += hx;
            s->fy[v] += hy;
            double w[9];
            long idx[9];
            orc_ib_weights(s, s->x[v], s->y[v], w, idx);
            double Ux = 0.0, Uy = 0.0;
            for (int q = 0; q < 9; ++q) {
                if (idx[q] < 0) continue;
                double pq, uq, vq;
                flow_at(s, idx[q], &pq, &uq, &vq);
                Ux += w[q] * uq;
                Uy += w[q] * vq;
            }
            double aLx = s->x[v] - s->x[L], aLy = s->y[v] - s->y[L];
            double aRx = s->x[R] - s->x[v], aRy = s->y[R] - s->y[v];
            double dV = 0.5 * (sqrt(aLx * aLx + aLy * aLy) + sqrt(aRx * aRx + aRy * aRy));
            s->ibx[v] = 2.0 * dV * (s->vx[v] - Ux);
            s->iby[v] = 2.0 * dV * (s->vy[v] - Uy);
        }
        free(fe);
    }
}

/* Eqs. verletPos and verletVel for a deformable particle: each vertex moves
 * by the interpolated fluid velocity U_v (the first tentative velocity) plus
 * half its acceleration F_v / m_v, m_v = rho_P A_0 / n (the particle's mass
 * spread evenly over its vertices); its velocity is the second-order backward
 * difference 3/2 x^{n+1} - 2 x^n + 1/2 x^{n-1}, written as
 * 3/2 (x^{n+1} - x^n) - 1/2 (x^n - x^{n-1}) (first-order on the first step). */
static void soft_advance(orc_sim *s, int m, long step) {
    int off = s->mem_off[m], n = s->mem_n[m];
    double mv = s->mem_rhop[m] * s->mem_A0[m] / n;
    for (int v = off; v < off + n; ++v) {
        double xn = s->x[v] + (s->Ux[v] + 0.5 * s->fx[v] / mv);
        double yn = s->y[v] + (s->Uy[v] + 0.5 * s->fy[v] / mv);
        if (step == 0) {
            s->vx[v] = xn - s->x[v];
            s->vy[v] = yn - s->y[v];
        } else {
            s->vx[v] = 1.5 * (xn - s->x[v]) - 0.5 * (s->x[v] - s->xp[v]);
            s->vy[v] = 1.5 * (yn - s->y[v]) - 0.5 * (s->y[v] - s->yp[v]);
        }
        s->xp[v] = s->x[v];
        s->yp[v] = s->y[v];
        s->x[v] = xn;
        s->y[v] = yn;
    }
}

/* Eqs. linearVelRig and angularVelRig for a rigid particle: the total force F
 * and its moment M about the area centroid give du/dt = F/m and
 * domega/dt = M/I (m = rho_P A_0, I = rho_P J_0); u and omega advance by the
 * printed second-order form (forward Euler on the first step).  The body then
 * translates by u Delta t and turns by omega Delta t about its centroid, and
 * each vertex takes the rigid velocity u + omega x r.  cos(omega) - 1 is
 * formed as -2 sin^2(omega/2) (no cancellation for small turns). */
static void rigid_advance(orc_sim *s, int m, long step) {
    int off = s->mem_off[m], n = s->mem_n[m];
    double A, cx, cy, J;
    orc_ring_mass_properties(n, s->x + off, s->y + off, &A, &cx, &cy, &J);
    double x0 = s->x[off], y0 = s->y[off];
    double Fx = 0.0, Fy = 0.0, M = 0.0;
    for (int v = off; v < off + n; ++v) {
        double rx = (s->x[v] - x0) - cx, ry = (s->y[v] - y0) - cy;
        Fx += s->fx[v];
        Fy += s->fy[v];
        M += rx * s->fy[v] - ry * s->fx[v];
    }
    double mass = s->mem_rhop[m] * s->mem_A0[m], inertia = s->mem_rhop[m] * s->mem_J0[m];
    double ax = Fx / mass, ay = Fy / mass, al = M / inertia;
    double *rb = s->mem_rb + 6 * m;
    double un, vn, wn;
    if (step == 0) {
        un = rb[0] + ax;
        vn = rb[1] + ay;
        wn = rb[4] + al;
    } else {
        un = (2.0 / 3.0) * (2.0 * rb[0] - 0.5 * rb[2] + ax);
        vn = (2.0 / 3.0) * (2.0 * rb[1] - 0.5 * rb[3] + ay);
        wn = (2.0 / 3.0) * (2.0 * rb[4] - 0.5 * rb[5] + al);
    }
    rb[2] = rb[0]; rb[3] = rb[1]; rb[5] = rb[4];
    rb[0] = un; rb[1] = vn; rb[4] = wn;
    double h = sin(0.5 * wn);
    double c1 = -2.0 * h * h, sn = sin(wn);
    for (int v = off; v < off + n; ++v) {
        double rx = (s->x[v] - x0) - cx, ry = (s->y[v] - y0) - cy;
        double drx = c1 * rx - sn * ry, dry = sn * rx + c1 * ry;
        s->vx[v] = un - wn * (ry + dry);
        s->vy[v] = vn + wn * (rx + drx);
        s->xp[v] = s->x[v];
        s->yp[v] = s->y[v];
        s->x[v] = s->x[v] + (un + drx);
        s->y[v] = s->y[v] + (vn + dry);
    }
}

/* advance of every dynamic membrane from the total forces F_v and the
 * interpolated velocities U_v held in the state (step 10 for kinds 2, 3) */
void orc_particle_advance(orc_sim *s, long step) {
    for (int m = 0; m < s->nmem; ++m) {
        if (s->mem_kind[m] == 2) soft_advance(s, m, step);
        else if (s->mem_kind[m] == 3) rigid_advance(s, m, step);
    }
}

void orc_set_membrane_density(orc_sim *s, int m, double rho_p) { s->mem_rhop[m] = rho_p; }
double orc_membrane_inertia(const orc_sim *s, int m) { return s->mem_rhop[m] * s->mem_J0[m]; }
double orc_membrane_mass(const orc_sim *s, int m) { return s->mem_rhop[m] * s->mem_A0[m]; }

/* ------------------------------------------------------------------------- */
/* Simulation object                                                          */
/* ------------------------------------------------------------------------- */

orc_sim *orc_create(int nx, int ny, double tau, double gx, double gy, int walls) {
    orc_sim *s = (orc_sim *)calloc(1, sizeof(orc_sim));
    long N = (long)nx * ny;
    s->nx = nx; s->ny = ny; s->tau = tau; s->gx = gx; s->gy = gy; s->walls = walls;
    s->f = (double *)calloc(9 * N, sizeof(double));
    s->ftmp = (double *)calloc(9 * N, sizeof(double));
    s->rho = (double *)calloc(N, sizeof(double));
    s->ux = (double *)calloc(N, sizeof(double));
    s->uy = (double *)calloc(N, sizeof(double));
    s->Gx = (double *)calloc(N, sizeof(double));
    s->Gy = (double *)calloc(N, sizeof(double));
    for (int i = 0; i < 9; ++i)
        for (long n = 0; n < N; ++n) s->f[i * N + n] = W9[i];
    s->d_rep = 2.0;
    s->p_ref = 1.0 / 3.0;
    s->d_cut = 1.5; s->y_eq = 0.75; s->d_break = 3.0;
    return s;
}

void orc_destroy(orc_sim *s) {
    if (!s) return;
    free(s->f); free(s->ftmp); free(s->rho); free(s->ux); free(s->uy);
    free(s->Gx); free(s->Gy);
    free(s->mem_off); free(s->mem_n); free(s->mem_kind); free(s->mem_ks); free(s->mem_kb);
    free(s->mem_ka); free(s->mem_A0); free(s->vert_mem);
    free(s->x); free(s->y); free(s->xp); free(s->yp); free(s->fx); free(s->fy);
    free(s->l0); free(s->th0); free(s->wgt); free(s->widx); free(s->Ux); free(s->Uy);
    free(s->lig_elem); free(s->rx); free(s->ry); free(s->bond_of_lig); free(s->owner_of_rec);
    free(s->mem_rhop); free(s->mem_J0); free(s->mem_rb);
    free(s->vx); free(s->vy); free(s->hx); free(s->hy); free(s->ibx); free(s->iby);
    free(s);
}

void orc_set_populations(orc_sim *s, const double *f) {
    memcpy(s->f, f, sizeof(double) * 9 * (size_t)s->nx * s->ny);
}
void orc_get_populations(const orc_sim *s, double *f) {
    memcpy(f, s->f, sizeof(double) * 9 * (size_t)s->nx * s->ny);
}
void orc_get_fields(const orc_sim *s, double *rho, double *ux, double *uy) {
    size_t N = (size_t)s->nx * s->ny;
    memcpy(rho, s->rho, N * sizeof(double));
    memcpy(ux, s->ux, N * sizeof(double));
    memcpy(uy, s->uy, N * sizeof(double));
}
void orc_get_force_field(const orc_sim *s, double *gx, double *gy) {
    size_t N = (size_t)s->nx * s->ny;
    memcpy(gx, s->Gx, N * sizeof(double));
    memcpy(gy, s->Gy, N * sizeof(double));
}

/* Poiseuille start (Sec. 3 drive; tau = 1 discrete fixed point): post-collision
 * f* = feq(1, u(y)) + F(u(y), G) with u(y) = 3 G (y + 1/2)(NY - 1/2 - y) + G/4,
 * streamed once to give the pre-collision state f^0. */
void orc_init_poiseuille(orc_sim *s) {
    long nx = s->nx, ny = s->ny, N = nx * ny;
    double feq[9], F[9];
    double G = s->gx;
    double nu = (s->tau - 0.5) / 3.0;
    for (long y = 0; y < ny; ++y) {
        double yy = (double)y;
        double u = G / (2.0 * nu) * (yy + 0.5) * ((double)ny - 0.5 - yy) + 0.25 * G;
        orc_equilibrium(1.0, u, 0.0, feq);
        orc_guo_source(s->tau, u, 0.0, s->gx, s->gy, F);
        for (long x = 0; x < nx; ++x)
            for (int i = 0; i < 9; ++i) s->ftmp[i * N + y * nx + x] = feq[i] + F[i];
    }
    orc_stream(s, s->ftmp, s->f);
}

/* x velocities of the two walls (Couette set-up, Sec. 4: planar Couette flow
 * in the cell-free layer) */
void orc_set_wall_velocity(orc_sim *s, double u_bottom, double u_top) {
    s->uw_bot = u_bottom;
    s->uw_top = u_top;
}

/* tau = 1 planar Couette state between the walls: post-collision f* =
 * feq(1, u(y)) with u(y) = u_bot + (u_top - u_bot) (y + 1/2) / NY, streamed.
 * With tau = 1 this is the discrete steady state: the pulled populations have
 * density 1 and velocity u(y) (the quadratic terms of feq cancel for a linear
 * profile), and the moving-wall bounce-back reproduces the half-way walls. */
void orc_init_couette(orc_sim *s) {
    long nx = s->nx, ny = s->ny, N = nx * ny;
    double feq[9];
    for (long y = 0; y < ny; ++y) {
        double u = s->uw_bot + (s->uw_top - s->uw_bot) * ((double)y + 0.5) / (double)ny;
        orc_equilibrium(1.0, u, 0.0, feq);
        for (long x = 0; x < nx; ++x)
            for (int i = 0; i < 9; ++i) s->ftmp[i * N + y * nx + x] = feq[i];
    }
    orc_stream(s, s->ftmp, s->f);
}

static void *grow(void *p, size_t n, size_t sz) { return realloc(p, n * sz); }

/* add a closed CCW ring of n vertices, rest shape = given positions.
 * kind 0: kinematic (Eq. kinematicPos); kind 1: velocities projected on a rigid
 * motion before the advance; kind 2: dynamic deformable particle (Eqs.
 * newtonSoft, verletPos, verletVel); kind 3: dynamic rigid particle (Eqs.
 * linearVelRig, angularVelRig). ligand_elems are local element ids. */
int orc_add_membrane(orc_sim *s, const double *xy, int n, double ks, double kb, double ka,
                     int kind, const int *ligand_elems, int nlig) {
    int m = s->nmem++;
    int off = s->nv;
    int nv = s->nv + n;
    s->mem_off = grow(s->mem_off, s->nmem, sizeof(int));
    s->mem_n = grow(s->mem_n, s->nmem, sizeof(int));
    s->mem_kind = grow(s->mem_kind, s->nmem, sizeof(int));
    s->mem_ks = grow(s->mem_ks, s->nmem, sizeof(double));
    s->mem_kb = grow(s->mem_kb, s->nmem, sizeof(double));
    s->mem_ka = grow(s->mem_ka, s->nmem, sizeof(double));
    s->mem_A0 = grow(s->mem_A0, s->nmem, sizeof(double));
    s->vert_mem = grow(s->vert_mem, nv, sizeof(int));
    s->x = grow(s->x, nv, sizeof(double)); s->y = grow(s->y, nv, sizeof(double));
    s->xp = grow(s->xp, nv, sizeof(double)); s->yp = grow(s->yp, nv, sizeof(double));
    s->fx = grow(s->fx, nv, sizeof(double)); s->fy = grow(s->fy, nv, sizeof(double));
    s->l0 = grow(s->l0, nv, sizeof(double)); s->th0 = grow(s->th0, nv, sizeof(double));
    s->Ux = grow(s->Ux, nv, sizeof(double)); s->Uy = grow(s->Uy, nv, sizeof(double));
    s->wgt = grow(s->wgt, (size_t)nv * 9, sizeof(double));
    s->widx = grow(s->widx, (size_t)nv * 9, sizeof(long));
    s->mem_rhop = grow(s->mem_rhop, s->nmem, sizeof(double));
    s->mem_J0 = grow(s->mem_J0, s->nmem, sizeof(double));
    s->mem_rb = grow(s->mem_rb, (size_t)s->nmem * 6, sizeof(double));
    s->vx = grow(s->vx, nv, sizeof(double)); s->vy = grow(s->vy, nv, sizeof(double));
    s->hx = grow(s->hx, nv, sizeof(double)); s->hy = grow(s->hy, nv, sizeof(double));
    s->ibx = grow(s->ibx, nv, sizeof(double)); s->iby = grow(s->iby, nv, sizeof(double));
    s->mem_off[m] = off; s->mem_n[m] = n; s->mem_kind[m] = kind;
    s->mem_ks[m] = ks; s->mem_kb[m] = kb; s->mem_ka[m] = ka;
    for (int v = 0; v < n; ++v) {
        s->x[off + v] = xy[2 * v];
        s->y[off + v] = xy[2 * v + 1];
        s->xp[off + v] = xy[2 * v];
        s->yp[off + v] = xy[2 * v + 1];
        s->fx[off + v] = 0.0; s->fy[off + v] = 0.0;
        s->Ux[off + v] = 0.0; s->Uy[off + v] = 0.0;
        s->vx[off + v] = 0.0; s->vy[off + v] = 0.0;  /* particles start at rest (Sec. 3) */
        s->hx[off + v] = 0.0; s->hy[off + v] = 0.0;
        s->ibx[off + v] = 0.0; s->iby[off + v] = 0.0;
        s->vert_mem[off + v] = m;
    }
    orc_ring_rest(n, s->x + off, s->y + off, s->l0 + off, s->th0 + off, &s->mem_A0[m]);
    for (int k = 0; k < 6; ++k) s->mem_rb[6 * m + k] = 0.0;
    {
        double A, cx, cy;
        orc_ring_mass_properties(n, s->x + off, s->y + off, &A, &cx, &cy, &s->mem_J0[m]);
    }
    s->mem_rhop[m] = 1.1;  /* rho_P / rho = 1.1 (Sec. 3) */
    s->nv = nv;
    if (nlig > 0) {
        s->lig_elem = grow(s->lig_elem, s->nlig + nlig, sizeof(int));
        s->bond_of_lig = grow(s->bond_of_lig, s->nlig + nlig, sizeof(int));
        for (int k = 0; k < nlig; ++k) {
            s->lig_elem[s->nlig + k] = off + ligand_elems[k];
            s->bond_of_lig[s->nlig + k] = -1;
        }
        s->nlig += nlig;
    }
    return m;
}

void orc_set_receptors(orc_sim *s, const double *xy, int n, double d_cut, double y_eq,
                       double sigma, double kf_dt, double kr0_dt, double beta_f,
                       double beta_r, double d_break, uint64_t seed, uint64_t instance) {
    s->nrec = n;
    s->rx = grow(s->rx, n > 0 ? n : 1, sizeof(double));
    s->ry = grow(s->ry, n > 0 ? n : 1, sizeof(double));
    s->owner_of_rec = grow(s->owner_of_rec, n > 0 ? n : 1, sizeof(int));
    for (int r = 0; r < n; ++r) {
        s->rx[r] = xy[2 * r];
        s->ry[r] = xy[2 * r + 1];
        s->owner_of_rec[r] = -1;
    }
    s->d_cut = d_cut; s->y_eq = y_eq; s->sigma = sigma;
    s->kf_dt = kf_dt; s->kr0_dt = kr0_dt; s->beta_f = beta_f; s->beta_r = beta_r;
    s->d_break = d_break; s->seed = seed; s->instance = instance;
}

void orc_set_repulsion(orc_sim *s, double d_rep) { s->d_rep = d_rep; }

/* x distance with the periodic minimum image (and y when y is periodic) */
static void min_image(const orc_sim *s, double *dx, double *dy) {
    *dx -= s->nx * floor(*dx / s->nx + 0.5);
    if (!s->walls) *dy -= s->ny * floor(*dy / s->ny + 0.5);
}

/* ligand point: centroid of its element (Sec. 2.2, wall-particle interaction) */
static void ligand_point(const orc_sim *s, int l, double *cx, double *cy) {
    int a = s->lig_elem[l];
    int m = s->vert_mem[a];
    int b = s->mem_off[m] + (a - s->mem_off[m] + 1) % s->mem_n[m];
    *cx = 0.5 * (s->x[a] + s->x[b]);
    *cy = 0.5 * (s->y[a] + s->y[b]);
}

static double ligand_receptor_dist(const orc_sim *s, int l, int r, double *ddx, double *ddy) {
    double cx, cy;
    ligand_point(s, l, &cx, &cy);
    double dx = s->rx[r] - cx, dy = s->ry[r] - cy;
    min_image(s, &dx, &dy);
    if (ddx) *ddx = dx;
    if (ddy) *ddy = dy;
    return sqrt(dx * dx + dy * dy);
}

/* forward (formation) and reverse (rupture) probabilities per step */
double orc_p_form(const orc_sim *s, double d) {
    double z = (d - s->y_eq) / s->y_eq;
    return 1.0 - exp(-s->kf_dt * exp(-s->beta_f * z * z));
}
double orc_p_rupture(const orc_sim *s, double d) {
    double z = (d - s->y_eq) / s->y_eq;
    return 1.0 - exp(-s->kr0_dt * exp(s->beta_r * z * z));
}

/* steps 1-5: all Lagrangian forces at X^n */
void orc_compute_forces(orc_sim *s) {
    int nv = s->nv;
    for (int v = 0; v < nv; ++v) { s->fx[v] = 0.0; s->fy[v] = 0.0; }
    /* 1. bonds, Eq. adhFor, along ligand->receptor, half to each end vertex */
    for (int l = 0; l < s->nlig; ++l) {
        int r = s->bond_of_lig[l];
        if (r < 0) continue;
        double dx, dy;
        double d = ligand_receptor_dist(s, l, r, &dx, &dy);
        double c = s->sigma * (d - s->y_eq) / d;
        int a = s->lig_elem[l];
        int m = s->vert_mem[a];
        int b = s->mem_off[m] + (a - s->mem_off[m] + 1) % s->mem_n[m];
        s->fx[a] += 0.5 * c * dx; s->fy[a] += 0.5 * c * dy;
        s->fx[b] += 0.5 * c * dx; s->fy[b] += 0.5 * c * dy;
    }
    /* 2. repulsion, Eq. repFor (Delta x = 1), along the vertex's inward normal */
    if (s->nmem > 1) {
        const double c0 = 1e-4 / (8.0 * sqrt(2.0));
#pragma omp parallel for schedule(dynamic, 16)
        for (int a = 0; a < nv; ++a) {
            int ma = s->vert_mem[a];
            int off = s->mem_off[ma], n = s->mem_n[ma];
            double th, nvx, nvy, lL, lR;
            vertex_geometry(n, s->x + off, s->y + off, a - off, &th, &nvx, &nvy, &lL, &lR);
            for (int b = 0; b < nv; ++b) {
                if (s->vert_mem[b] == ma) continue;
                double dx = s->x[a] - s->x[b], dy = s->y[a] - s->y[b];
                min_image(s, &dx, &dy);
                double d = sqrt(dx * dx + dy * dy);
                if (d < s->d_rep) {
                    double mag = c0 * sqrt(1.0 / (d * d * d * d * d));
                    s->fx[a] -= mag * nvx;
                    s->fy[a] -= mag * nvy;
                }
            }
        }
    }
    /* 3-5. stretch, bend, area per ring */
    for (int m = 0; m < s->nmem; ++m) {
        int off = s->mem_off[m], n = s->mem_n[m];
        orc_ring_forces(n, s->x + off, s->y + off, s->l0 + off, s->th0 + off, s->mem_A0[m],
                        s->mem_ks[m], s->mem_kb[m], s->mem_ka[m], s->p_ref, 7,
                        s->fx + off, s->fy + off);
    }
}

/* step 11: rupture, then formation (lowest ligand id wins a receptor) */
void orc_bonds_update(orc_sim *s, long step) {
    int *was_free = (int *)malloc(sizeof(int) * (s->nrec > 0 ? s->nrec : 1));
    int *claimed = (int *)malloc(sizeof(int) * (s->nrec > 0 ? s->nrec : 1));
    for (int r = 0; r < s->nrec; ++r) {
        was_free[r] = s->owner_of_rec[r] < 0;
        claimed[r] = 0;
    }
    for (int l = 0; l < s->nlig; ++l) {
        int r = s->bond_of_lig[l];
        if (r < 0) continue;
        double d = ligand_receptor_dist(s, l, r, NULL, NULL);
        int rupture = d >= s->d_break;
        if (!rupture) rupture = orc_uniform(s->seed, s->instance, step, l, r, 1) < orc_p_rupture(s, d);
        if (rupture) {
            s->bond_of_lig[l] = -1;
            s->owner_of_rec[r] = -1;
        }
    }
    for (int l = 0; l < s->nlig; ++l) {
        if (s->bond_of_lig[l] >= 0) continue;
        for (int r = 0; r < s->nrec; ++r) {
            if (!was_free[r]) continue;
            double d = ligand_receptor_dist(s, l, r, NULL, NULL);
            if (!(d < s->d_cut)) continue;
            if (orc_uniform(s->seed, s->instance, step, l, r, 0) < orc_p_form(s, d)) {
                /* first accepted receptor is this ligand's candidate */
                if (!claimed[r]) {
                    claimed[r] = 1;
                    s->bond_of_lig[l] = r;
                    s->owner_of_rec[r] = l;
                }
                break;
            }
        }
    }
    free(was_free);
    free(claimed);
}

/* steps 1-5 and, for dynamic membranes, their hydrodynamic forces and the
 * forces they exert on the fluid */
void orc_compute_step_forces(orc_sim *s) {
    orc_compute_forces(s);
    dynamic_coupling(s);
}

/* one full step n -> n+1 */
static void step_once(orc_sim *s) {
    long N = (long)s->nx * s->ny;
    int nv = s->nv;
    orc_compute_step_forces(s);
    /* 6. weights at X^n */
#pragma omp parallel for schedule(static)
    for (int v = 0; v < nv; ++v) orc_ib_weights(s, s->x[v], s->y[v], s->wgt + 9 * v, s->widx + 9 * v);
    /* 7. spread: the membrane forces of kinematic membranes, the forcing
     * term F^ib of dynamic ones */
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) { s->Gx[n] = s->gx; s->Gy[n] = s->gy; }
    for (int v = 0; v < nv; ++v) {
        int dyn = is_dynamic(s->mem_kind[s->vert_mem[v]]);
        double Fx = dyn ? s->ibx[v] : s->fx[v], Fy = dyn ? s->iby[v] : s->fy[v];
        for (int k = 0; k < 9; ++k) {
            long j = s->widx[9 * v + k];
            if (j < 0) continue;
            s->Gx[j] += s->wgt[9 * v + k] * Fx;
            s->Gy[j] += s->wgt[9 * v + k] * Fy;
        }
    }
    /* 8. collide + stream */
    collide_and_stream(s);
    /* 9. interpolate u^n at X^n */
#pragma omp parallel for schedule(static)
    for (int v = 0; v < nv; ++v) {
        double a = 0.0, b = 0.0;
        for (int k = 0; k < 9; ++k) {
            long j = s->widx[9 * v + k];
            if (j < 0) continue;
            a += s->wgt[9 * v + k] * s->ux[j];
            b += s->wgt[9 * v + k] * s->uy[j];
        }
        s->Ux[v] = a;
        s->Uy[v] = b;
    }
    /* 10. advance (rigid projection first for kind 1; Newton for kinds 2, 3) */
    orc_particle_advance(s, s->step);
    for (int m = 0; m < s->nmem; ++m) {
        int off = s->mem_off[m], n = s->mem_n[m];
        if (is_dynamic(s->mem_kind[m])) continue;
        if (s->mem_kind[m] == 1) {
            double xc = 0, yc = 0, uc = 0, vc = 0;
            for (int v = off; v < off + n; ++v) { xc += s->x[v]; yc += s->y[v]; uc += s->Ux[v]; vc += s->Uy[v]; }
            xc /= n; yc /= n; uc /= n; vc /= n;
            double num = 0, den = 0;
            for (int v = off; v < off + n; ++v) {
                double rx = s->x[v] - xc, ry = s->y[v] - yc;
                num += rx * (s->Uy[v] - vc) - ry * (s->Ux[v] - uc);
                den += rx * rx + ry * ry;
            }
            double om = num / den;
            for (int v = off; v < off + n; ++v) {
                double rx = s->x[v] - xc, ry = s->y[v] - yc;
                s->Ux[v] = uc - om * ry;
                s->Uy[v] = vc + om * rx;
            }
        }
        for (int v = off; v < off + n; ++v) {
            double xn, yn;
            if (s->step == 0) {
                xn = s->x[v] + s->Ux[v];
                yn = s->y[v] + s->Uy[v];
            } else {
                xn = (2.0 / 3.0) * (2.0 * s->x[v] - 0.5 * s->xp[v] + s->Ux[v]);
                yn = (2.0 / 3.0) * (2.0 * s->y[v] - 0.5 * s->yp[v] + s->Uy[v]);
            }
            s->xp[v] = s->x[v]; s->yp[v] = s->y[v];
            s->x[v] = xn; s->y[v] = yn;
        }
    }
    /* 11. bonds at X^{n+1}, counter n */
    if (s->nlig > 0 && s->nrec > 0) orc_bonds_update(s, s->step);
    s->step += 1;
}

void orc_step(orc_sim *s, long nsteps) {
    for (long k = 0; k < nsteps; ++k) step_once(s);
}

/* threads of the OpenMP build (the plain build ignores the pragmas above,
 * whose loops write disjoint elements, so both builds give the same bits) */
#ifdef _OPENMP
#include <omp.h>
int orc_set_threads(int n) { if (n > 0) omp_set_num_threads(n); return omp_get_max_threads(); }
#else
int orc_set_threads(int n) { (void)n; return 1; }
#endif

/* accessors */
int orc_num_vertices(const orc_sim *s) { return s->nv; }
int orc_num_ligands(const orc_sim *s) { return s->nlig; }
long orc_get_step(const orc_sim *s) { return s->step; }
void orc_get_markers(const orc_sim *s, double *xy) {
    for (int v = 0; v < s->nv; ++v) { xy[2 * v] = s->x[v]; xy[2 * v + 1] = s->y[v]; }
}
void orc_get_prev_markers(const orc_sim *s, double *xy) {
    for (int v = 0; v < s->nv; ++v) { xy[2 * v] = s->xp[v]; xy[2 * v + 1] = s->yp[v]; }
}
void orc_set_markers(orc_sim *s, const double *xy, const double *xy_prev) {
    for (int v = 0; v < s->nv; ++v) {
        s->x[v] = xy[2 * v]; s->y[v] = xy[2 * v + 1];
        if (xy_prev) { s->xp[v] = xy_prev[2 * v]; s->yp[v] = xy_prev[2 * v + 1]; }
    }
}
void orc_get_forces(const orc_sim *s, double *fxy) {
    for (int v = 0; v < s->nv; ++v) { fxy[2 * v] = s->fx[v]; fxy[2 * v + 1] = s->fy[v]; }
}
void orc_get_marker_velocity(const orc_sim *s, double *uxy) {
    for (int v = 0; v < s->nv; ++v) { uxy[2 * v] = s->Ux[v]; uxy[2 * v + 1] = s->Uy[v]; }
}
void orc_set_forces(orc_sim *s, const double *fxy) {
    for (int v = 0; v < s->nv; ++v) { s->fx[v] = fxy[2 * v]; s->fy[v] = fxy[2 * v + 1]; }
}
void orc_set_marker_velocity(orc_sim *s, const double *uxy) {
    for (int v = 0; v < s->nv; ++v) { s->Ux[v] = uxy[2 * v]; s->Uy[v] = uxy[2 * v + 1]; }
}
void orc_get_particle_velocity(const orc_sim *s, double *vxy) {
    for (int v = 0; v < s->nv; ++v) { vxy[2 * v] = s->vx[v]; vxy[2 * v + 1] = s->vy[v]; }
}
void orc_set_particle_velocity(orc_sim *s, const double *vxy) {
    for (int v = 0; v < s->nv; ++v) { s->vx[v] = vxy[2 * v]; s->vy[v] = vxy[2 * v + 1]; }
}
void orc_get_hydro_forces(const orc_sim *s, double *fxy) {
    for (int v = 0; v < s->nv; ++v) { fxy[2 * v] = s->hx[v]; fxy[2 * v + 1] = s->hy[v]; }
}
void orc_get_ib_forces(const orc_sim *s, double *fxy) {
    for (int v = 0; v < s->nv; ++v) { fxy[2 * v] = s->ibx[v]; fxy[2 * v + 1] = s->iby[v]; }
}
void orc_get_rigid_state(const orc_sim *s, int m, double *out) {
    for (int k = 0; k < 6; ++k) out[k] = s->mem_rb[6 * m + k];
}
/* set the rigid state (u, v, u_prev, v_prev, omega, omega_prev) of a rigid
 * dynamic membrane and the matching vertex velocities u + omega x r (r from
 * the area centroid) */
void orc_set_rigid_state(orc_sim *s, int m, const double *in) {
    int off = s->mem_off[m], n = s->mem_n[m];
    for (int k = 0; k < 6; ++k) s->mem_rb[6 * m + k] = in[k];
    double A, cx, cy, J;
    orc_ring_mass_properties(n, s->x + off, s->y + off, &A, &cx, &cy, &J);
    for (int v = off; v < off + n; ++v) {
        double rx = (s->x[v] - s->x[off]) - cx, ry = (s->y[v] - s->y[off]) - cy;
        s->vx[v] = in[0] - in[4] * ry;
        s->vy[v] = in[1] + in[4] * rx;
    }
}
void orc_get_bonds(const orc_sim *s, int *bond_of_lig) {
    for (int l = 0; l < s->nlig; ++l) bond_of_lig[l] = s->bond_of_lig[l];
}
void orc_set_bond(orc_sim *s, int l, int r) {
    if (s->bond_of_lig[l] >= 0) s->owner_of_rec[s->bond_of_lig[l]] = -1;
    s->bond_of_lig[l] = r;
    if (r >= 0) s->owner_of_rec[r] = l;
}
double orc_mass(const orc_sim *s) {
    long N = (long)s->nx * s->ny;
    double m = 0.0;
    for (long k = 0; k < 9 * N; ++k) m += s->f[k];
    return m;
}
double orc_membrane_area(const orc_sim *s, int m) {
    return orc_ring_area(s->mem_n[m], s->x + s->mem_off[m], s->y + s->mem_off[m]);
}
double orc_membrane_rest_area(const orc_sim *s, int m) { return s->mem_A0[m]; }

/* ========================================================================= */
/* Forward-mode tangent of the step (FP64 dual numbers v + d eps, eps^2 = 0)  */
/*                                                                           */
/* The derivative of steps 1-10 above along one direction of (k_s, k_b per    */
/* membrane, sigma, X^n, X^{n-1}, f^n), each step differentiated as written   */
/* above, with every branch (stencil origin, dropped wall rows, repulsion     */
/* range, minimum image) taken at the primal value.  Bond events (step 11)    */
/* are not differentiated: the tangent runs along the primal's bond history.  */
/* Kinematic membranes only (no rigid projection).                            */
/* ========================================================================= */
typedef struct {
    double v, d;
} dn;

static dn dn_make(double v, double d) {
    dn r;
    r.v = v;
    r.d = d;
    return r;
}
static dn dn_c(double v) { return dn_make(v, 0.0); }
static dn dn_add(dn a, dn b) { return dn_make(a.v + b.v, a.d + b.d); }
static dn dn_sub(dn a, dn b) { return dn_make(a.v - b.v, a.d - b.d); }
static dn dn_neg(dn a) { return dn_make(-a.v, -a.d); }
static dn dn_scale(double c, dn a) { return dn_make(c * a.v, c * a.d); }
static dn dn_mul(dn a, dn b) { return dn_make(a.v * b.v, a.d * b.v + a.v * b.d); }
/* (a/b)' = (a' - (a/b) b') / b */
static dn dn_div(dn a, dn b) {
    double q = a.v / b.v;
    return dn_make(q, (a.d - q * b.d) / b.v);
}
/* sqrt(a)' = a' / (2 sqrt(a)) */
static dn dn_sqrt(dn a) {
    double r = sqrt(a.v);
    return dn_make(r, a.d / (2.0 * r));
}
/* atan2(y, x)' = (x y' - y x') / (x^2 + y^2) */
static dn dn_atan2(dn y, dn x) {
    return dn_make(atan2(y.v, x.v), (x.v * y.d - y.v * x.d) / (x.v * x.v + y.v * y.v));
}
static dn dn_fabs(dn a) { return a.v < 0.0 ? dn_neg(a) : a; }

typedef struct {
    orc_sim *s;                  /* primal (not owned) */
    long N;
    double *df, *dftmp;          /* tangent of the pre-collision f^n, scratch */
    double *dx, *dy, *dxp, *dyp; /* tangent of X^n and X^{n-1} */
    double *dks, *dkb;           /* tangent of k_s, k_b per membrane */
    double dsigma;               /* tangent of the bond stiffness */
    dn *Fx, *Fy;                 /* [nv] force */
    dn *W;                       /* [nv][9] shape functions */
    long *idx;                   /* [nv][9] node of each (-1: dropped) */
    dn *Gx, *Gy;                 /* [N] force field */
    dn *ux, *uy;                 /* [N] velocity of the collide */
} orc_tangent;

static dn t_x(const orc_tangent *t, int v) { return dn_make(t->s->x[v], t->dx[v]); }
static dn t_y(const orc_tangent *t, int v) { return dn_make(t->s->y[v], t->dy[v]); }

/* vertex_geometry on dual positions (ring of n vertices starting at off) */
static void t_vertex_geometry(const orc_tangent *t, int off, int n, int v, dn *theta, dn *nvx, dn *nvy,
                              dn *lL, dn *lR) {
    int L = off + (v + n - 1) % n, C = off + v, R = off + (v + 1) % n;
    dn eLx = dn_sub(t_x(t, C), t_x(t, L)), eLy = dn_sub(t_y(t, C), t_y(t, L));
    dn eRx = dn_sub(t_x(t, R), t_x(t, C)), eRy = dn_sub(t_y(t, R), t_y(t, C));
    dn a = dn_sqrt(dn_add(dn_mul(eLx, eLx), dn_mul(eLy, eLy)));
    dn b = dn_sqrt(dn_add(dn_mul(eRx, eRx), dn_mul(eRy, eRy)));
    dn cr = dn_sub(dn_mul(eLx, eRy), dn_mul(eLy, eRx));
    dn dt = dn_add(dn_mul(eLx, eRx), dn_mul(eLy, eRy));
    *theta = dn_atan2(cr, dt);
    dn nx_ = dn_add(dn_div(eLy, a), dn_div(eRy, b));
    dn ny_ = dn_sub(dn_neg(dn_div(eLx, a)), dn_div(eRx, b));
    dn nn = dn_sqrt(dn_add(dn_mul(nx_, nx_), dn_mul(ny_, ny_)));
    *nvx = dn_div(nx_, nn);
    *nvy = dn_div(ny_, nn);
    *lL = a;
    *lR = b;
}

/* shoelace area about vertex 0, on dual positions */
static dn t_ring_area(const orc_tangent *t, int off, int n) {
    dn s = dn_c(0.0);
    dn xr = t_x(t, off), yr = t_y(t, off);
    for (int v = 0; v < n; ++v) {
        int a = off + v, b = off + (v + 1) % n;
        s = dn_add(s, dn_sub(dn_mul(dn_sub(t_x(t, a), xr), dn_sub(t_y(t, b), yr)),
                             dn_mul(dn_sub(t_x(t, b), xr), dn_sub(t_y(t, a), yr))));
    }
    return dn_scale(0.5, s);
}

/* steps 3-5 (Eqs. strainFor, bendFor, areaFor) of membrane m on duals */
static void t_ring_forces(orc_tangent *t, int m) {
    orc_sim *s = t->s;
    int off = s->mem_off[m], n = s->mem_n[m];
    dn ks = dn_make(s->mem_ks[m], t->dks[m]), kb = dn_make(s->mem_kb[m], t->dkb[m]);
    for (int v = 0; v < n; ++v) {
        int a = off + v, b = off + (v + 1) % n;
        dn rx = dn_sub(t_x(t, a), t_x(t, b)), ry = dn_sub(t_y(t, a), t_y(t, b));
        dn l = dn_sqrt(dn_add(dn_mul(rx, rx), dn_mul(ry, ry)));
        dn c = dn_div(dn_mul(dn_neg(ks), dn_sub(l, dn_c(s->l0[a]))), l);
        t->Fx[a] = dn_add(t->Fx[a], dn_mul(c, rx));
        t->Fy[a] = dn_add(t->Fy[a], dn_mul(c, ry));
        t->Fx[b] = dn_sub(t->Fx[b], dn_mul(c, rx));
        t->Fy[b] = dn_sub(t->Fy[b], dn_mul(c, ry));
    }
    for (int v = 0; v < n; ++v) {
        int L = off + (v + n - 1) % n, C = off + v, R = off + (v + 1) % n;
        dn th, nvx, nvy, lL, lR;
        t_vertex_geometry(t, off, n, v, &th, &nvx, &nvy, &lL, &lR);
        dn mo = dn_mul(kb, dn_sub(th, dn_c(s->th0[C])));
        dn sL = dn_div(lL, dn_add(lL, lR)), sR = dn_div(lR, dn_add(lL, lR));
        t->Fx[L] = dn_add(t->Fx[L], dn_mul(dn_mul(mo, sL), nvx));
        t->Fy[L] = dn_add(t->Fy[L], dn_mul(dn_mul(mo, sL), nvy));
        t->Fx[C] = dn_sub(t->Fx[C], dn_mul(mo, nvx));
        t->Fy[C] = dn_sub(t->Fy[C], dn_mul(mo, nvy));
        t->Fx[R] = dn_add(t->Fx[R], dn_mul(dn_mul(mo, sR), nvx));
        t->Fy[R] = dn_add(t->Fy[R], dn_mul(dn_mul(mo, sR), nvy));
    }
    dn A = t_ring_area(t, off, n);
    dn c = dn_scale(s->p_ref, dn_scale(-s->mem_ka[m], dn_sub(dn_c(1.0), dn_div(A, dn_c(s->mem_A0[m])))));
    for (int v = 0; v < n; ++v) {
        int a = off + v, b = off + (v + 1) % n;
        dn ex = dn_sub(t_x(t, b), t_x(t, a)), ey = dn_sub(t_y(t, b), t_y(t, a));
        dn Fx = dn_mul(c, dn_neg(ey)), Fy = dn_mul(c, ex);
        t->Fx[a] = dn_add(t->Fx[a], dn_scale(0.5, Fx));
        t->Fy[a] = dn_add(t->Fy[a], dn_scale(0.5, Fy));
        t->Fx[b] = dn_add(t->Fx[b], dn_scale(0.5, Fx));
        t->Fy[b] = dn_add(t->Fy[b], dn_scale(0.5, Fy));
    }
}

/* steps 1-5 on duals (orc_compute_forces differentiated) */
static void t_compute_forces(orc_tangent *t) {
    orc_sim *s = t->s;
    int nv = s->nv;
    for (int v = 0; v < nv; ++v) {
        t->Fx[v] = dn_c(0.0);
        t->Fy[v] = dn_c(0.0);
    }
    /* 1. bonds (Eq. adhFor); the minimum-image shift is a constant */
    dn sigma = dn_make(s->sigma, t->dsigma);
    for (int l = 0; l < s->nlig; ++l) {
        int r = s->bond_of_lig[l];
        if (r < 0) continue;
        int a = s->lig_elem[l];
        int m = s->vert_mem[a];
        int b = s->mem_off[m] + (a - s->mem_off[m] + 1) % s->mem_n[m];
        dn cx = dn_scale(0.5, dn_add(t_x(t, a), t_x(t, b)));
        dn cy = dn_scale(0.5, dn_add(t_y(t, a), t_y(t, b)));
        dn dx = dn_sub(dn_c(s->rx[r]), cx), dy = dn_sub(dn_c(s->ry[r]), cy);
        double sx = dx.v, sy = dy.v;
        min_image(s, &sx, &sy);
        dx.v = sx;
        dy.v = sy;
        dn d = dn_sqrt(dn_add(dn_mul(dx, dx), dn_mul(dy, dy)));
        dn c = dn_div(dn_mul(sigma, dn_sub(d, dn_c(s->y_eq))), d);
        t->Fx[a] = dn_add(t->Fx[a], dn_scale(0.5, dn_mul(c, dx)));
        t->Fy[a] = dn_add(t->Fy[a], dn_scale(0.5, dn_mul(c, dy)));
        t->Fx[b] = dn_add(t->Fx[b], dn_scale(0.5, dn_mul(c, dx)));
        t->Fy[b] = dn_add(t->Fy[b], dn_scale(0.5, dn_mul(c, dy)));
    }
    /* 2. repulsion (Eq. repFor), pairs within d_rep at the primal distance */
    if (s->nmem > 1) {
        const double c0 = 1e-4 / (8.0 * sqrt(2.0));
        for (int a = 0; a < nv; ++a) {
            int ma = s->vert_mem[a];
            int off = s->mem_off[ma], n = s->mem_n[ma];
            dn th, nvx, nvy, lL, lR;
            t_vertex_geometry(t, off, n, a - off, &th, &nvx, &nvy, &lL, &lR);
            for (int b = 0; b < nv; ++b) {
                if (s->vert_mem[b] == ma) continue;
                dn dx = dn_sub(t_x(t, a), t_x(t, b)), dy = dn_sub(t_y(t, a), t_y(t, b));
                double sx = dx.v, sy = dy.v;
                min_image(s, &sx, &sy);
                dx.v = sx;
                dy.v = sy;
                dn d = dn_sqrt(dn_add(dn_mul(dx, dx), dn_mul(dy, dy)));
                if (d.v < s->d_rep) {
                    dn d5 = dn_mul(dn_mul(dn_mul(dn_mul(d, d), d), d), d);
                    dn mag = dn_scale(c0, dn_sqrt(dn_div(dn_c(1.0), d5)));
                    t->Fx[a] = dn_sub(t->Fx[a], dn_mul(mag, nvx));
                    t->Fy[a] = dn_sub(t->Fy[a], dn_mul(mag, nvy));
                }
            }
        }
    }
    /* 3-5 */
    for (int m = 0; m < s->nmem; ++m) t_ring_forces(t, m);
}

/* Roma kernel on a dual argument */
static dn t_roma(dn r) {
    dn a = dn_fabs(r);
    if (a.v <= 0.5) return dn_scale(1.0 / 3.0, dn_add(dn_c(1.0), dn_sqrt(dn_sub(dn_c(1.0), dn_scale(3.0, dn_mul(a, a))))));
    if (a.v <= 1.5) {
        dn b = dn_sub(dn_c(1.0), a);
        dn q = dn_sqrt(dn_sub(dn_c(1.0), dn_scale(3.0, dn_mul(b, b))));
        return dn_div(dn_sub(dn_sub(dn_c(5.0), dn_scale(3.0, a)), q), dn_c(6.0));
    }
    return dn_c(0.0);
}

/* orc_ib_weights on a dual point (same stencil, same dropped rows) */
static void t_ib_weights(const orc_sim *s, dn px, dn py, dn w[9], long idx[9]) {
    long i0 = (long)floor(px.v + 0.5), j0 = (long)floor(py.v + 0.5);
    dn Wr[9], rx[9], ry[9];
    int nvalid = 0;
    for (int b = -1; b <= 1; ++b) {
        for (int a = -1; a <= 1; ++a) {
            int k = (b + 1) * 3 + (a + 1);
            long i = i0 + a, j = j0 + b;
            rx[k] = dn_sub(dn_c((double)i), px);
            ry[k] = dn_sub(dn_c((double)j), py);
            int inside = s->walls ? (j >= 0 && j < s->ny) : 1;
            if (inside) {
                Wr[k] = dn_mul(t_roma(rx[k]), t_roma(ry[k]));
                idx[k] = imod(j, s->ny) * s->nx + imod(i, s->nx);
                ++nvalid;
            } else {
                Wr[k] = dn_c(0.0);
                idx[k] = -1;
            }
        }
    }
    if (nvalid == 9) {
        for (int k = 0; k < 9; ++k) w[k] = Wr[k];
        return;
    }
    dn A[3][3];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) A[r][c] = dn_c(0.0);
    dn sumW = dn_c(0.0);
    for (int k = 0; k < 9; ++k) {
        dn p[3] = {dn_c(1.0), rx[k], ry[k]};
        sumW = dn_add(sumW, Wr[k]);
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) A[r][c] = dn_add(A[r][c], dn_mul(dn_mul(Wr[k], p[r]), p[c]));
    }
    dn c00 = dn_sub(dn_mul(A[1][1], A[2][2]), dn_mul(A[1][2], A[2][1]));
    dn c10 = dn_neg(dn_sub(dn_mul(A[1][0], A[2][2]), dn_mul(A[1][2], A[2][0])));
    dn c20 = dn_sub(dn_mul(A[1][0], A[2][1]), dn_mul(A[1][1], A[2][0]));
    dn det = dn_add(dn_add(dn_mul(A[0][0], c00), dn_mul(A[0][1], c10)), dn_mul(A[0][2], c20));
    if (det.v > 1e-10) {
        dn cv[3] = {dn_div(c00, det), dn_div(c10, det), dn_div(c20, det)};
        for (int k = 0; k < 9; ++k)
            w[k] = dn_mul(Wr[k], dn_add(dn_add(cv[0], dn_mul(cv[1], rx[k])), dn_mul(cv[2], ry[k])));
    } else if (sumW.v > 0.0) {
        for (int k = 0; k < 9; ++k) w[k] = dn_div(Wr[k], sumW);
    } else {
        for (int k = 0; k < 9; ++k) w[k] = dn_c(0.0);
    }
}

/* steps 6-10 and the tangent of the populations, on duals; then the primal
 * step.  Reads the primal state of step n before step_once replaces it. */
static void t_step_once(orc_tangent *t) {
    orc_sim *s = t->s;
    long N = t->N;
    int nv = s->nv;
    t_compute_forces(t);
    /* 6. weights at X^n; 7. spread */
    for (int v = 0; v < nv; ++v) t_ib_weights(s, t_x(t, v), t_y(t, v), t->W + 9 * v, t->idx + 9 * v);
    for (long n = 0; n < N; ++n) {
        t->Gx[n] = dn_c(s->gx);
        t->Gy[n] = dn_c(s->gy);
    }
    for (int v = 0; v < nv; ++v)
        for (int k = 0; k < 9; ++k) {
            long j = t->idx[9 * v + k];
            if (j < 0) continue;
            t->Gx[j] = dn_add(t->Gx[j], dn_mul(t->W[9 * v + k], t->Fx[v]));
            t->Gy[j] = dn_add(t->Gy[j], dn_mul(t->W[9 * v + k], t->Fy[v]));
        }
    /* 8. collide (Eqs. feq, forcedBGK, ForcingTerm with rho u = sum f e + G/2) */
    double pre = 1.0 - 1.0 / (2.0 * s->tau);
    for (long n = 0; n < N; ++n) {
        dn f[9];
        for (int i = 0; i < 9; ++i) f[i] = dn_make(s->f[i * N + n], t->df[i * N + n]);
        dn r = dn_c(0.0), jx = dn_c(0.0), jy = dn_c(0.0);
        for (int i = 0; i < 9; ++i) {
            r = dn_add(r, f[i]);
            jx = dn_add(jx, dn_scale((double)EX[i], f[i]));
            jy = dn_add(jy, dn_scale((double)EY[i], f[i]));
        }
        dn gx = t->Gx[n], gy = t->Gy[n];
        jx = dn_add(jx, dn_scale(0.5, gx));
        jy = dn_add(jy, dn_scale(0.5, gy));
        dn ux = dn_div(jx, r), uy = dn_div(jy, r);
        t->ux[n] = ux;
        t->uy[n] = uy;
        dn uu = dn_add(dn_mul(ux, ux), dn_mul(uy, uy));
        for (int i = 0; i < 9; ++i) {
            dn eu = dn_add(dn_scale((double)EX[i], ux), dn_scale((double)EY[i], uy));
            dn feq = dn_scale(W9[i], dn_mul(r, dn_sub(dn_add(dn_add(dn_c(1.0), dn_scale(3.0, eu)),
                                                             dn_scale(4.5, dn_mul(eu, eu))),
                                                      dn_scale(1.5, uu))));
            dn cx = dn_add(dn_scale(3.0, dn_sub(dn_c((double)EX[i]), ux)), dn_scale(9.0 * EX[i], eu));
            dn cy = dn_add(dn_scale(3.0, dn_sub(dn_c((double)EY[i]), uy)), dn_scale(9.0 * EY[i], eu));
            dn F = dn_scale(pre * W9[i], dn_add(dn_mul(cx, gx), dn_mul(cy, gy)));
            dn out = dn_add(dn_sub(f[i], dn_scale(1.0 / s->tau, dn_sub(f[i], feq))), F);
            t->dftmp[i * N + n] = out.d;
        }
    }
    /* streaming of the tangent: the same permutation as the populations */
    orc_stream(s, t->dftmp, t->df);
    /* 9. interpolation; 10. BDF2 (Euler on step 0) */
    for (int v = 0; v < nv; ++v) {
        dn a = dn_c(0.0), b = dn_c(0.0);
        for (int k = 0; k < 9; ++k) {
            long j = t->idx[9 * v + k];
            if (j < 0) continue;
            a = dn_add(a, dn_mul(t->W[9 * v + k], t->ux[j]));
            b = dn_add(b, dn_mul(t->W[9 * v + k], t->uy[j]));
        }
        double nx_, ny_;
        if (s->step == 0) {
            nx_ = t->dx[v] + a.d;
            ny_ = t->dy[v] + b.d;
        } else {
            nx_ = (2.0 / 3.0) * (2.0 * t->dx[v] - 0.5 * t->dxp[v] + a.d);
            ny_ = (2.0 / 3.0) * (2.0 * t->dy[v] - 0.5 * t->dyp[v] + b.d);
        }
        t->dxp[v] = t->dx[v];
        t->dyp[v] = t->dy[v];
        t->dx[v] = nx_;
        t->dy[v] = ny_;
    }
    step_once(s);
}

/* Tangent object.  Returns NULL if a membrane is rigid-projected. */
orc_tangent *orc_tangent_create(orc_sim *s) {
    for (int m = 0; m < s->nmem; ++m)
        if (s->mem_kind[m] != 0) return NULL;
    orc_tangent *t = (orc_tangent *)calloc(1, sizeof(orc_tangent));
    long N = (long)s->nx * s->ny;
    int nv = s->nv > 0 ? s->nv : 1, nm = s->nmem > 0 ? s->nmem : 1;
    t->s = s;
    t->N = N;
    t->df = (double *)calloc(9 * N, sizeof(double));
    t->dftmp = (double *)calloc(9 * N, sizeof(double));
    t->dx = (double *)calloc(nv, sizeof(double));
    t->dy = (double *)calloc(nv, sizeof(double));
    t->dxp = (double *)calloc(nv, sizeof(double));
    t->dyp = (double *)calloc(nv, sizeof(double));
    t->dks = (double *)calloc(nm, sizeof(double));
    t->dkb = (double *)calloc(nm, sizeof(double));
    t->Fx = (dn *)calloc(nv, sizeof(dn));
    t->Fy = (dn *)calloc(nv, sizeof(dn));
    t->W = (dn *)calloc(9 * (size_t)nv, sizeof(dn));
    t->idx = (long *)calloc(9 * (size_t)nv, sizeof(long));
    t->Gx = (dn *)calloc(N, sizeof(dn));
    t->Gy = (dn *)calloc(N, sizeof(dn));
    t->ux = (dn *)calloc(N, sizeof(dn));
    t->uy = (dn *)calloc(N, sizeof(dn));
    return t;
}

void orc_tangent_destroy(orc_tangent *t) {
    if (!t) return;
    free(t->df); free(t->dftmp); free(t->dx); free(t->dy); free(t->dxp); free(t->dyp);
    free(t->dks); free(t->dkb); free(t->Fx); free(t->Fy); free(t->W); free(t->idx);
    free(t->Gx); free(t->Gy); free(t->ux); free(t->uy);
    free(t);
}

/* direction: dks, dkb [nmem] (NULL = 0), dsigma, dxy / dxy_prev [nv][2]
 * (NULL = 0; dxy_prev NULL = dxy), df [9][ny][nx] of the pre-collision
 * populations (NULL = 0) */
void orc_tangent_seed(orc_tangent *t, const double *dks, const double *dkb, double dsigma, const double *dxy,
                      const double *dxy_prev, const double *df) {
    orc_sim *s = t->s;
    for (int m = 0; m < s->nmem; ++m) {
        t->dks[m] = dks ? dks[m] : 0.0;
        t->dkb[m] = dkb ? dkb[m] : 0.0;
    }
    t->dsigma = dsigma;
    const double *pv = dxy_prev ? dxy_prev : dxy;
    for (int v = 0; v < s->nv; ++v) {
        t->dx[v] = dxy ? dxy[2 * v] : 0.0;
        t->dy[v] = dxy ? dxy[2 * v + 1] : 0.0;
        t->dxp[v] = pv ? pv[2 * v] : 0.0;
        t->dyp[v] = pv ? pv[2 * v + 1] : 0.0;
    }
    for (long k = 0; k < 9 * t->N; ++k) t->df[k] = df ? df[k] : 0.0;
}

/* n primal steps with their tangent */
void orc_tangent_step(orc_tangent *t, long n) {
    for (long k = 0; k < n; ++k) t_step_once(t);
}

void orc_tangent_get(const orc_tangent *t, double *dxy, double *dxy_prev, double *df) {
    const orc_sim *s = t->s;
    for (int v = 0; v < s->nv; ++v) {
        if (dxy) { dxy[2 * v] = t->dx[v]; dxy[2 * v + 1] = t->dy[v]; }
        if (dxy_prev) { dxy_prev[2 * v] = t->dxp[v]; dxy_prev[2 * v + 1] = t->dyp[v]; }
    }
    if (df) memcpy(df, t->df, sizeof(double) * 9 * t->N);
}
