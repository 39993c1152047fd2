/*
 * capfilm oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, double-precision CPU restatement of the coupled lattice
 * Boltzmann / FEM capsule method of Wouters, Aouane, Sega & Harting,
 * "Capillary interactions between soft capsules protruding through thin fluid
 * films" (Sec. 3.1 "Method description", Sec. 3.2 "Simulation setup").
 * Only tests/, the smoke check and the CPU-baseline leg of the benchmark may
 * load this library; the product path never does.  It shares no code, header
 * or table with the CUDA library.
 *
 * One time step, in the order the method describes it:
 *   1. streaming with half-way bounce-back on the substrate and on lattice links
 *      cut by membrane elements, with Ladd's moving-wall term and the momentum
 *      exchanged with each element (Sec. 3.1, coupling paragraph)
 *   2. moments rho^c = sum_i f_i^c, j^c = sum_i f_i^c e_i (Eq. 4 context)
 *   3. pseudopotential psi^c = 1 - exp(-rho^c) and the Shan-Chen force (Eq. 10),
 *      with the interior/exterior decoupling: across a cut link (or into the
 *      substrate) the partner density is interpolated from the node's own side
 *      and the reaction goes to the crossed element (Sec. 3.1, last paragraph)
 *   4. BGK collision towards the 2nd-order equilibrium (Eqs. 4-5), with the
 *      Shan-Chen velocity-shift forcing
 *   5. element forces averaged over two consecutive steps, spread with equal
 *      weights to the three element nodes (Sec. 3.1, homogeneous scheme)
 *   6. membrane forces: Skalak strain (Eq. 6), Helfrich bending (Eq. 7),
 *      volume penalty (Eq. 8), Hertz repulsion (Eq. 11); node update
 *      x(t+1) = x(t) + F_tot/m (Eq. 9)
 *   7. new cut links for the moved membrane.
 * An optional drying step (a reading: the paper fixes each film height per
 * run and lowers none) follows the collision, see remove_mass below.
 * The flag OR_IBM replaces the cut-link parts of steps 1, 3 and 5 and the node
 * update of step 6 with a diffuse-interface (immersed-boundary) coupling, a
 * variant that is not part of the paper: the membrane forces are spread with
 * Peskin's 4-point kernel, act on the fluid in the collision, and the nodes
 * move with the interpolated fluid velocity.
 * Points where the paper is silent are resolved the same way as in the CUDA
 * library and are listed as readings c1..c25 in the design notes.
 *
 * Every function below is pinned, against closed forms, invariants and brute
 * force, by the tests/test_oracle_*.py files.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <float.h>

#define NQ 19
#define MAXCAPS 256

/* D3Q19 velocity set and weights (Sec. 3.1, below Eq. 5): w0 = 1/3, six
 * nearest neighbours 1/18, twelve diagonal neighbours 1/36.  Opposite
 * directions are stored as pairs (1,2), (3,4), ... so opp(i) = i^1 shifted. */
static const int EV[NQ][3] = {
    {0, 0, 0},
    {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
    {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
    {1, 0, 1}, {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1}, {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
static double WV[NQ];
static int wv_ready = 0;
static void init_weights(void) {
    if (wv_ready) return;
    WV[0] = 1.0 / 3.0;
    for (int i = 1; i <= 6; ++i) WV[i] = 1.0 / 18.0;
    for (int i = 7; i < NQ; ++i) WV[i] = 1.0 / 36.0;
    wv_ready = 1;
}
static int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
static const double CS2 = 1.0 / 3.0;

/* ------------------------------------------------------------------ types */
typedef struct {
    int nv, nf, mode;
    double kS, C, kB, kV, mass;
    double *X, *V, *Xref;       /* [nv*3] positions, velocities, reference */
    int *F;                     /* [nf*3] faces, outward orientation       */
    double *refM;               /* [nf*3] inverse reference metric m11,m12,m22 */
    double *refA;               /* [nf]   reference area                   */
    double *refDet;             /* [nf]   det of reference metric          */
    double V0;                  /* reference volume                       */
    double *FT_prev, *FT_cur;   /* [nf*3] element momentum exchange       */
    double *Fcpl, *Fel, *Fint, *Ftot; /* [nv*3] node forces of the last step */
    double force[3];            /* sum of coupling forces (last step)     */
    double torque[3];
    double area, volume;
    double wet;                 /* wetting offset of the interpolated densities */
    int tri_base;               /* global index of face 0                 */
} or_capsule;

typedef struct or_ctx {
    int nx, ny, nz, wall;
    long N;
    double tau[2], G, zrep, delta0, xi;
    double *fpost, *fpre;       /* [2][19][N] */
    double *rho, *u;            /* [2][N], [3][N] recorded each step        */
    uint32_t *mask;             /* [N] bit (k-1): link x -> x+e_k is cut   */
    int *tri;                   /* [N*18] crossing element per cut link    */
    uint8_t *inside;            /* [N] capsule interior flag (column parity) */
    double *slink;              /* [N*18] scalar exchange per cut link     */
    int ncaps, ntri;
    or_capsule caps[MAXCAPS];
    long step;
    double dmA;                 /* drying: A mass turned into B per step (0: off) */
    int flags;                  /* alternative readings (OR_* below)       */
    double *fibm;               /* [3][N] spread membrane force (OR_IBM)   */
    double mom_to_membrane[3];  /* cumulative momentum given to membranes  */
    double mom_to_wall[3];      /* cumulative momentum given to substrate  */
} or_ctx;

/* Alternative readings of points where the paper is silent (the defaults
 * are the readings c6, c8, c10, c23 of the design notes):
 *   OR_INERTIAL  node update v += F/m, x += v instead of x += F/m (c6)
 *   OR_REF_RHO   Ladd's term with the reference density rho_0 = 1 instead
 *                of the node's density (c8)
 *   OR_MIRROR    partner density across a cut or substrate link = the node's
 *                own density instead of the mean over its side (c10)
 *   OR_REMOVE    drying removes the A mass instead of turning it into B (c23) */
enum { OR_INERTIAL = 1, OR_REF_RHO = 2, OR_MIRROR = 4, OR_REMOVE = 8, OR_IBM = 16 };
/*   OR_IBM      diffuse-interface (immersed-boundary) coupling instead of the
 *               cut-link bounce-back: the membrane forces are spread to the
 *               lattice with Peskin's 4-point kernel and enter the collision
 *               as a body force shared by the components in proportion to
 *               their densities; the nodes move with the fluid velocity
 *               interpolated with the same kernel; no link is cut for the
 *               fluid (the cut structure is kept for the interior flags). */

/* cut bits the lattice sees: none with the diffuse-interface coupling */
static uint32_t lmask(const or_ctx *c, long n) { return (c->flags & OR_IBM) ? 0u : c->mask[n]; }

static long nidx(const or_ctx *c, int x, int y, int z) {
    return ((long)z * c->ny + y) * c->nx + x;
}
static int wrap(int a, int n) { a %= n; return a < 0 ? a + n : a; }
static int is_solid(const or_ctx *c, int z) { return c->wall && z == 0; }
static double *F_(or_ctx *c, double *base, int comp, int i, long n) {
    return &base[((long)comp * NQ + i) * c->N + n];
}

/* ------------------------------------------------------ equilibrium (Eq. 5) */
static void equilibrium(double rho, const double u[3], double feq[NQ]) {
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < NQ; ++i) {
        double eu = EV[i][0] * u[0] + EV[i][1] * u[1] + EV[i][2] * u[2];
        feq[i] = WV[i] * rho * (1.0 + eu / CS2 - uu / (2.0 * CS2) + eu * eu / (2.0 * CS2 * CS2));
    }
}

static double psi_of(double rho) { return 1.0 - exp(-rho); }  /* Sec. 3.1, below Eq. 10 */

/* ------------------------------------------------------------- creation */
or_ctx *or_create(int nx, int ny, int nz, int wall, double tauA, double tauB, double G,
                  double rep_dz) {
    init_weights();
    or_ctx *c = (or_ctx *)calloc(1, sizeof(or_ctx));
    c->nx = nx; c->ny = ny; c->nz = nz; c->wall = wall;
    c->N = (long)nx * ny * nz;
    c->tau[0] = tauA; c->tau[1] = tauB; c->G = G;
    c->zrep = 0.5 + rep_dz; c->delta0 = 1.5; c->xi = 1.5;  /* Sec. 3.2, Eq. 11 */
    c->fpost = (double *)calloc(2 * NQ * c->N, sizeof(double));
    c->fpre = (double *)calloc(2 * NQ * c->N, sizeof(double));
    c->rho = (double *)calloc(2 * c->N, sizeof(double));
    c->u = (double *)calloc(3 * c->N, sizeof(double));
    c->mask = (uint32_t *)calloc(c->N, sizeof(uint32_t));
    c->tri = (int *)malloc(sizeof(int) * 18 * c->N);
    c->slink = (double *)calloc(18 * c->N, sizeof(double));
    c->inside = (uint8_t *)calloc(c->N, 1);
    for (long k = 0; k < 18 * c->N; ++k) c->tri[k] = -1;
    return c;
}

void or_destroy(or_ctx *c) {
    if (!c) return;
    for (int k = 0; k < c->ncaps; ++k) {
        or_capsule *p = &c->caps[k];
        free(p->X); free(p->V); free(p->Xref); free(p->F); free(p->refM); free(p->refA);
        free(p->refDet); free(p->FT_prev); free(p->FT_cur); free(p->Fcpl); free(p->Fel);
        free(p->Fint); free(p->Ftot);
    }
    free(c->fpost); free(c->fpre); free(c->rho); free(c->u); free(c->mask); free(c->tri);
    free(c->slink); free(c->inside); free(c->fibm);
    free(c);
}

/* --------------------------------------------------- vector helpers */
static void sub3(const double *a, const double *b, double *o) { o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2]; }
static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double *a, const double *b, double *o) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}
static double norm3(const double *a) { return sqrt(dot3(a, a)); }

/* ---------------------------------------------- membrane energies/forces */
/* Reference state of the Skalak law: for each face the metric of the
 * stress-free triangle, G0 = [[U1.U1, U1.U2],[U1.U2, U2.U2]] with U1, U2 the
 * reference edge vectors from the first node; we keep G0^-1 and det G0. */
static void reference_state(const double *X, const int *F, int nf, double *refM,
                            double *refA, double *refDet) {
    for (int f = 0; f < nf; ++f) {
        const double *a = &X[3 * F[3 * f]], *b = &X[3 * F[3 * f + 1]], *cc = &X[3 * F[3 * f + 2]];
        double U1[3], U2[3], n[3];
        sub3(b, a, U1); sub3(cc, a, U2);
        double g11 = dot3(U1, U1), g12 = dot3(U1, U2), g22 = dot3(U2, U2);
        double det = g11 * g22 - g12 * g12;
        refM[3 * f] = g22 / det; refM[3 * f + 1] = -g12 / det; refM[3 * f + 2] = g11 / det;
        refDet[f] = det;
        cross3(U1, U2, n);
        refA[f] = 0.5 * norm3(n);
    }
}

/* Skalak strain energy (Eq. 6) on linear triangles.  The squared principal
 * stretches are the eigenvalues of G0^-1 g, so I1 = tr(G0^-1 g) - 2 and
 * I2 = det g / det G0 - 1.  E_face = A0 kS/4 (I1^2 + 2 I1 - 2 I2 + C I2^2).
 * Forces are the exact negative gradient (virtual work). Returns energy. */
static double skalak(const double *X, const int *F, int nf, const double *refM,
                     const double *refA, const double *refDet, double kS, double C,
                     double *Fout) {
    double E = 0.0;
    for (int f = 0; f < nf; ++f) {
        int ia = F[3 * f], ib = F[3 * f + 1], ic = F[3 * f + 2];
        double u1[3], u2[3];
        sub3(&X[3 * ib], &X[3 * ia], u1); sub3(&X[3 * ic], &X[3 * ia], u2);
        double g11 = dot3(u1, u1), g12 = dot3(u1, u2), g22 = dot3(u2, u2);
        double m11 = refM[3 * f], m12 = refM[3 * f + 1], m22 = refM[3 * f + 2];
        double I1 = m11 * g11 + 2.0 * m12 * g12 + m22 * g22 - 2.0;
        double I2 = (g11 * g22 - g12 * g12) / refDet[f] - 1.0;
        double A0 = refA[f];
        E += A0 * kS / 4.0 * (I1 * I1 + 2.0 * I1 - 2.0 * I2 + C * I2 * I2);
        if (!Fout) continue;
        double dW1 = kS / 4.0 * (2.0 * I1 + 2.0);
        double dW2 = kS / 4.0 * (-2.0 + 2.0 * C * I2);
        double gb[3], gc[3];
        for (int k = 0; k < 3; ++k) {
            double dI1_u1 = 2.0 * (m11 * u1[k] + m12 * u2[k]);
            double dI1_u2 = 2.0 * (m12 * u1[k] + m22 * u2[k]);
            double dI2_u1 = 2.0 * (g22 * u1[k] - g12 * u2[k]) / refDet[f];
            double dI2_u2 = 2.0 * (g11 * u2[k] - g12 * u1[k]) / refDet[f];
            gb[k] = A0 * (dW1 * dI1_u1 + dW2 * dI2_u1);
            gc[k] = A0 * (dW1 * dI1_u2 + dW2 * dI2_u2);
        }
        for (int k = 0; k < 3; ++k) {
            Fout[3 * ib + k] -= gb[k];
            Fout[3 * ic + k] -= gc[k];
            Fout[3 * ia + k] += gb[k] + gc[k];
        }
    }
    return E;
}

/* cot of the angle at o between edges o->p and o->q, and its gradient with
 * respect to p and q (the gradient w.r.t. o is minus their sum). */
static double cot_angle(const double *o, const double *p, const double *q, double dp[3], double dq[3]) {
    double u[3], w[3], n[3];
    sub3(p, o, u); sub3(q, o, w);
    cross3(u, w, n);
    double s = norm3(n), d = dot3(u, w);
    double uu = dot3(u, u), ww = dot3(w, w);
    if (dp) {
        for (int k = 0; k < 3; ++k) {
            double ds_du = (ww * u[k] - d * w[k]) / s;
            double ds_dw = (uu * w[k] - d * u[k]) / s;
            dp[k] = w[k] / s - d / (s * s) * ds_du;
            dq[k] = u[k] / s - d / (s * s) * ds_dw;
        }
    }
    return d / s;
}

/* Helfrich bending (Eq. 7) with H0 = 0 on the triangulated surface.  The mean
 * curvature normal at node v is the cotangent Laplacian divided by twice the
 * node area: 2H n = L_v / (2 A_v), L_v = sum_j (cot a_vj + cot b_vj)(x_j - x_v),
 * A_v = one third of the adjacent face areas.  E = kB/8 sum_v |L_v|^2 / A_v
 * (= kB/2 sum_v (2H_v)^2 A_v; 8 pi kB for a sphere).  The Gaussian term is a
 * topological constant on a closed surface and exerts no force.  Forces are the
 * exact negative gradient (the functional derivative of the discrete energy). */
static double helfrich(const double *X, const int *F, int nv, int nf, double kB, double *Fout) {
    double *L = (double *)calloc(3 * nv, sizeof(double));
    double *Av = (double *)calloc(nv, sizeof(double));
    for (int f = 0; f < nf; ++f) {
        int ia = F[3 * f], ib = F[3 * f + 1], ic = F[3 * f + 2];
        const double *a = &X[3 * ia], *b = &X[3 * ib], *c = &X[3 * ic];
        double cta = cot_angle(a, b, c, NULL, NULL);
        double ctb = cot_angle(b, c, a, NULL, NULL);
        double ctc = cot_angle(c, a, b, NULL, NULL);
        double u[3], w[3], n[3];
        sub3(b, a, u); sub3(c, a, w); cross3(u, w, n);
        double Af = 0.5 * norm3(n);
        for (int k = 0; k < 3; ++k) {
            L[3 * ia + k] += ctc * (b[k] - a[k]) + ctb * (c[k] - a[k]);
            L[3 * ib + k] += cta * (c[k] - b[k]) + ctc * (a[k] - b[k]);
            L[3 * ic + k] += ctb * (a[k] - c[k]) + cta * (b[k] - c[k]);
        }
        Av[ia] += Af / 3.0; Av[ib] += Af / 3.0; Av[ic] += Af / 3.0;
    }
    double E = 0.0;
    for (int v = 0; v < nv; ++v) E += kB / 8.0 * dot3(&L[3 * v], &L[3 * v]) / Av[v];
    if (Fout) {
        double *gL = (double *)malloc(sizeof(double) * 3 * nv);
        double *gA = (double *)malloc(sizeof(double) * nv);
        for (int v = 0; v < nv; ++v) {
            for (int k = 0; k < 3; ++k) gL[3 * v + k] = kB / 4.0 * L[3 * v + k] / Av[v];
            gA[v] = -kB / 8.0 * dot3(&L[3 * v], &L[3 * v]) / (Av[v] * Av[v]);
        }
        for (int f = 0; f < nf; ++f) {
            int ia = F[3 * f], ib = F[3 * f + 1], ic = F[3 * f + 2];
            const double *a = &X[3 * ia], *b = &X[3 * ib], *c = &X[3 * ic];
            double dA_b[3], dA_c[3];   /* cot derivatives reuse buffers below */
            double da_p[3], da_q[3], db_p[3], db_q[3], dc_p[3], dc_q[3];
            double cta = cot_angle(a, b, c, da_p, da_q);   /* p=b, q=c */
            double ctb = cot_angle(b, c, a, db_p, db_q);   /* p=c, q=a */
            double ctc = cot_angle(c, a, b, dc_p, dc_q);   /* p=a, q=b */
            const double *gLa = &gL[3 * ia], *gLb = &gL[3 * ib], *gLc = &gL[3 * ic];
            double ba[3], cb[3], ca[3];
            sub3(b, a, ba); sub3(c, b, cb); sub3(c, a, ca);
            double dga[3], dgb[3], dgc[3];
            sub3(gLb, gLc, dga); sub3(gLa, gLc, dgb); sub3(gLa, gLb, dgc);
            double gam_a = dot3(dga, cb);   /* coefficient of d(cot a) */
            double gam_b = dot3(dgb, ca);   /* coefficient of d(cot b) */
            double gam_c = dot3(dgc, ba);   /* coefficient of d(cot c) */
            /* face area gradient */
            double u[3], w[3], n[3];
            sub3(b, a, u); sub3(c, a, w); cross3(u, w, n);
            double s = norm3(n), d = dot3(u, w), uu = dot3(u, u), ww = dot3(w, w);
            for (int k = 0; k < 3; ++k) {
                dA_b[k] = 0.5 * (ww * u[k] - d * w[k]) / s;
                dA_c[k] = 0.5 * (uu * w[k] - d * u[k]) / s;
            }
            double gAf = (gA[ia] + gA[ib] + gA[ic]) / 3.0;
            for (int k = 0; k < 3; ++k) {
                double ga = 0.0, gb = 0.0, gc = 0.0;
                /* explicit edge-vector terms with cotangents held fixed */
                ga += ctc * (gLb[k] - gLa[k]) + ctb * (gLc[k] - gLa[k]);
                gb += ctc * (gLa[k] - gLb[k]) + cta * (gLc[k] - gLb[k]);
                gc += ctb * (gLa[k] - gLc[k]) + cta * (gLb[k] - gLc[k]);
                /* cot(a): o=a, p=b, q=c */
                gb += gam_a * da_p[k]; gc += gam_a * da_q[k]; ga -= gam_a * (da_p[k] + da_q[k]);
                /* cot(b): o=b, p=c, q=a */
                gc += gam_b * db_p[k]; ga += gam_b * db_q[k]; gb -= gam_b * (db_p[k] + db_q[k]);
                /* cot(c): o=c, p=a, q=b */
                ga += gam_c * dc_p[k]; gb += gam_c * dc_q[k]; gc -= gam_c * (dc_p[k] + dc_q[k]);
                /* node areas */
                gb += gAf * dA_b[k]; gc += gAf * dA_c[k]; ga -= gAf * (dA_b[k] + dA_c[k]);
                Fout[3 * ia + k] -= ga;
                Fout[3 * ib + k] -= gb;
                Fout[3 * ic + k] -= gc;
            }
        }
        free(gL); free(gA);
    }
    free(L); free(Av);
    return E;
}

/* Enclosed volume of a closed, outward-oriented mesh (divergence theorem). */
static double mesh_volume(const double *X, const int *F, int nf) {
    double V = 0.0;
    for (int f = 0; f < nf; ++f) {
        double n[3];
        cross3(&X[3 * F[3 * f + 1]], &X[3 * F[3 * f + 2]], n);
        V += dot3(&X[3 * F[3 * f]], n) / 6.0;
    }
    return V;
}

static double mesh_area(const double *X, const int *F, int nf) {
    double A = 0.0;
    for (int f = 0; f < nf; ++f) {
        double u[3], w[3], n[3];
        sub3(&X[3 * F[3 * f + 1]], &X[3 * F[3 * f]], u);
        sub3(&X[3 * F[3 * f + 2]], &X[3 * F[3 * f]], w);
        cross3(u, w, n);
        A += 0.5 * norm3(n);
    }
    return A;
}

/* Volume penalty (Eq. 8): E = kV/2 (V-V0)^2/V0, F_a = -kV (V-V0)/V0 dV/dx_a with
 * dV/dx_a = (x_b x x_c)/6 summed over the faces (a,b,c) containing a. */
static double volume_penalty(const double *X, const int *F, int nf, double kV, double V0,
                             double *Fout) {
    double V = mesh_volume(X, F, nf);
    double E = kV / 2.0 * (V - V0) * (V - V0) / V0;
    if (Fout) {
        double pre = -kV * (V - V0) / V0 / 6.0;
        for (int f = 0; f < nf; ++f) {
            int ia = F[3 * f], ib = F[3 * f + 1], ic = F[3 * f + 2];
            double na[3], nb[3], nc[3];
            cross3(&X[3 * ib], &X[3 * ic], na);
            cross3(&X[3 * ic], &X[3 * ia], nb);
            cross3(&X[3 * ia], &X[3 * ib], nc);
            for (int k = 0; k < 3; ++k) {
                Fout[3 * ia + k] += pre * na[k];
                Fout[3 * ib + k] += pre * nb[k];
                Fout[3 * ic + k] += pre * nc[k];
            }
        }
    }
    return E;
}

/* Hertz repulsion (Eq. 11), reading: overlap delta0 - d with d the node-node
 * (different capsules) or node-plane distance, F = Xi (delta0 - d)^1.5 along
 * the separation, acting only while d < delta0. */
static double hertz_mag(double xi, double delta0, double d) {
    double o = delta0 - d;
    return xi * o * sqrt(o);
}

/* ------------------------------------------------------------ cut links */
/* Orientation of d relative to the plane (a,b,c): det[b-a; c-a; d-a]. */
static double orient3(const double *a, const double *b, const double *c, const double *d) {
    double r1[3], r2[3], r3[3], n[3];
    sub3(b, a, r1); sub3(c, a, r2); sub3(d, a, r3);
    cross3(r2, r3, n);
    return dot3(r1, n);
}

/* Does the lattice link segment p->q cross triangle (A,B,C)?  Sign convention
 * sign(0) = +, so a segment through a shared edge is counted once.  Inputs are
 * single-precision node positions promoted to double; the decision is taken on
 * the same single-precision positions as the CUDA path stores. */
static int seg_tri(const double *p, const double *q, const double *A, const double *B,
                   const double *C) {
    double dp = orient3(A, B, C, p), dq = orient3(A, B, C, q);
    if ((dp >= 0.0) == (dq >= 0.0)) return 0;
    double s1 = orient3(p, q, A, B), s2 = orient3(p, q, B, C), s3 = orient3(p, q, C, A);
    return ((s1 >= 0.0) == (s2 >= 0.0)) && ((s2 >= 0.0) == (s3 >= 0.0));
}

static void clear_cuts(or_ctx *c) {
    memset(c->mask, 0, sizeof(uint32_t) * c->N);
    for (long k = 0; k < 18 * c->N; ++k) c->tri[k] = -1;
}

static void mark_link(or_ctx *c, int x, int y, int z, int k, int T) {
    long a = nidx(c, wrap(x, c->nx), wrap(y, c->ny), wrap(z, c->nz));
    int x2 = x + EV[k][0], y2 = y + EV[k][1], z2 = z + EV[k][2];
    long b = nidx(c, wrap(x2, c->nx), wrap(y2, c->ny), wrap(z2, c->nz));
    int kb = opp(k);
    /* a link is cut when it crosses the membrane an odd number of times, i.e.
     * when its end nodes lie on different sides: crossings toggle the bit */
    c->mask[a] ^= 1u << (k - 1);
    c->mask[b] ^= 1u << (kb - 1);
    if (c->tri[18 * a + k - 1] < 0 || T < c->tri[18 * a + k - 1]) c->tri[18 * a + k - 1] = T;
    if (c->tri[18 * b + kb - 1] < 0 || T < c->tri[18 * b + kb - 1]) c->tri[18 * b + kb - 1] = T;
}

/* the nine "positive" directions: each lattice link counted once */
static const int POS[9] = {1, 3, 5, 7, 9, 11, 13, 15, 17};

static void tri_vertices_f(const or_capsule *p, int f, double A[3], double B[3], double C[3]) {
    for (int k = 0; k < 3; ++k) {
        A[k] = (double)(float)p->X[3 * p->F[3 * f] + k];
        B[k] = (double)(float)p->X[3 * p->F[3 * f + 1] + k];
        C[k] = (double)(float)p->X[3 * p->F[3 * f + 2] + k];
    }
}

static int link_fluid(const or_ctx *c, int z, int k) {
    int z2 = z + EV[k][2];
    if (c->wall && (wrap(z, c->nz) == 0 || wrap(z2, c->nz) == 0)) return 0;
    return 1;
}

/* Cut links by enumerating, for each element, the lattice links inside its
 * bounding box (a link touching the element must start within one lattice
 * unit of the box).  A link is cut when the number of elements it crosses is
 * odd; its element is the smallest global index among those it crosses. */
/* Returns -1 (the cut structure left partial) when an element spans more than
 * 16 lattice units along an axis or has a non-finite vertex: a diverged
 * membrane, which the search below would otherwise walk without end. */
static int compute_cuts(or_ctx *c) {
    clear_cuts(c);
    for (int ci = 0; ci < c->ncaps; ++ci) {
        or_capsule *p = &c->caps[ci];
        for (int f = 0; f < p->nf; ++f) {
            double A[3], B[3], C[3];
            tri_vertices_f(p, f, A, B, C);
            int lo[3], hi[3];
            for (int k = 0; k < 3; ++k) {
                double mn = fmin(A[k], fmin(B[k], C[k])), mx = fmax(A[k], fmax(B[k], C[k]));
                if (!(mx - mn <= 16.0) || !isfinite(mn) || !isfinite(mx)) return -1;
                lo[k] = (int)ceil(mn - 1.0);
                hi[k] = (int)floor(mx + 1.0);
            }
            for (int z = lo[2]; z <= hi[2]; ++z)
                for (int y = lo[1]; y <= hi[1]; ++y)
                    for (int x = lo[0]; x <= hi[0]; ++x)
                        for (int d = 0; d < 9; ++d) {
                            int k = POS[d];
                            if (!link_fluid(c, z, k)) continue;
                            double P[3] = {x, y, z};
                            double Q[3] = {x + EV[k][0], y + EV[k][1], z + EV[k][2]};
                            if (seg_tri(P, Q, A, B, C)) mark_link(c, x, y, z, k, p->tri_base + f);
                        }
        }
    }
    return 0;
}

/* Interior flags by parity of cut +z links walked up each column. */
static void compute_inside(or_ctx *c) {
    for (int y = 0; y < c->ny; ++y)
        for (int x = 0; x < c->nx; ++x) {
            int in = 0;
            for (int z = 0; z < c->nz; ++z) {
                long n = nidx(c, x, y, z);
                c->inside[n] = (uint8_t)in;
                if (c->mask[n] & (1u << (5 - 1))) in ^= 1;
            }
        }
}

/* --------------------------------------------------------------- set-up */
int or_add_capsule(or_ctx *c, int nv, const double *X, int nf, const int *F, double kS,
                   double C, double kB, double kV, double mass, int mode) {
    if (c->ncaps >= MAXCAPS) return -1;
    or_capsule *p = &c->caps[c->ncaps];
    memset(p, 0, sizeof(*p));
    p->nv = nv; p->nf = nf; p->mode = mode;
    p->kS = kS; p->C = C; p->kB = kB; p->kV = kV; p->mass = mass;
    p->X = (double *)malloc(sizeof(double) * 3 * nv);
    p->Xref = (double *)malloc(sizeof(double) * 3 * nv);
    p->V = (double *)calloc(3 * nv, sizeof(double));
    p->F = (int *)malloc(sizeof(int) * 3 * nf);
    /* the stored state is single precision in the kernel: start from the same values */
    for (int k = 0; k < 3 * nv; ++k) p->X[k] = p->Xref[k] = (double)(float)X[k];
    memcpy(p->F, F, sizeof(int) * 3 * nf);
    p->refM = (double *)malloc(sizeof(double) * 3 * nf);
    p->refA = (double *)malloc(sizeof(double) * nf);
    p->refDet = (double *)malloc(sizeof(double) * nf);
    reference_state(p->Xref, p->F, nf, p->refM, p->refA, p->refDet);
    p->V0 = mesh_volume(p->Xref, p->F, nf);
    p->FT_prev = (double *)calloc(3 * nf, sizeof(double));
    p->FT_cur = (double *)calloc(3 * nf, sizeof(double));
    p->Fcpl = (double *)calloc(3 * nv, sizeof(double));
    p->Fel = (double *)calloc(3 * nv, sizeof(double));
    p->Fint = (double *)calloc(3 * nv, sizeof(double));
    p->Ftot = (double *)calloc(3 * nv, sizeof(double));
    p->tri_base = c->ntri;
    c->ntri += nf;
    p->area = mesh_area(p->X, p->F, nf);
    p->volume = p->V0;
    c->ncaps++;
    if (compute_cuts(c) != 0) return -1;
    compute_inside(c);
    return c->ncaps - 1;
}

/* Film set-up (Sec. 3.2): component A (index 0) below the film top, B above,
 * majority/minority densities rho_maj/rho_min, one mixed layer at rho_mix for
 * both components in the plane floor(h_top + 1/2); capsule interiors hold the
 * B-majority state; jitter [2][N] (may be NULL) is added to both densities.
 * Populations start at rest, f_i = w_i rho. */
int or_set_film(or_ctx *c, double h_top, double rho_maj, double rho_min, double rho_mix,
                const double *jit) {
    int zm = (int)floor(h_top + 0.5);
    for (int z = 0; z < c->nz; ++z)
        for (int y = 0; y < c->ny; ++y)
            for (int x = 0; x < c->nx; ++x) {
                long n = nidx(c, x, y, z);
                double r[2];
                if (is_solid(c, z)) { r[0] = r[1] = 0.0; }
                else {
                    if (c->inside[n]) { r[0] = rho_min; r[1] = rho_maj; }
                    else if (z < zm) { r[0] = rho_maj; r[1] = rho_min; }
                    else if (z == zm) { r[0] = rho_mix; r[1] = rho_mix; }
                    else { r[0] = rho_min; r[1] = rho_maj; }
                    if (jit) { r[0] += jit[n]; r[1] += jit[c->N + n]; }
                }
                for (int cc = 0; cc < 2; ++cc)
                    for (int i = 0; i < NQ; ++i) *F_(c, c->fpost, cc, i, n) = WV[i] * r[cc];
            }
    return 0;
}

/* Arbitrary post-collision populations (unit tests). */
void or_set_populations(or_ctx *c, const double *f) {
    memcpy(c->fpost, f, sizeof(double) * 2 * NQ * c->N);
}
void or_get_populations(const or_ctx *c, double *f) {
    memcpy(f, c->fpost, sizeof(double) * 2 * NQ * c->N);
}

/* ------------------------------------------------------------- the step */
static void uT_of(const or_ctx *c, int T, double uT[3]) {
    int ci = 0;
    while (ci + 1 < c->ncaps && c->caps[ci + 1].tri_base <= T) ++ci;
    const or_capsule *p = &c->caps[ci];
    int f = T - p->tri_base;
    for (int k = 0; k < 3; ++k)
        uT[k] = (p->V[3 * p->F[3 * f] + k] + p->V[3 * p->F[3 * f + 1] + k] + p->V[3 * p->F[3 * f + 2] + k]) / 3.0;
}

static or_capsule *capsule_of(or_ctx *c, int T, int *f) {
    int ci = 0;
    while (ci + 1 < c->ncaps && c->caps[ci + 1].tri_base <= T) ++ci;
    *f = T - c->caps[ci].tri_base;
    return &c->caps[ci];
}

static void stream(or_ctx *c) {
    long N = c->N;
    memset(c->slink, 0, sizeof(double) * 18 * N);
    double wallmom[3] = {0, 0, 0};
#pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < c->nz; ++z)
        for (int y = 0; y < c->ny; ++y)
            for (int x = 0; x < c->nx; ++x) {
                if (is_solid(c, z)) continue;
                long n = nidx(c, x, y, z);
                double rw[2] = {0, 0};
                for (int cc = 0; cc < 2; ++cc)
                    for (int j = 0; j < NQ; ++j) rw[cc] += *F_(c, c->fpost, cc, j, n);
                for (int i = 0; i < NQ; ++i) {
                    int sx = x - EV[i][0], sy = y - EV[i][1], sz = z - EV[i][2];
                    int ib = opp(i);  /* x + e_ib is the source node */
                    int solid = c->wall && wrap(sz, c->nz) == 0;
                    int cut = (i != 0) && (lmask(c, n) & (1u << (ib - 1)));
                    for (int cc = 0; cc < 2; ++cc) {
                        double *dst = F_(c, c->fpre, cc, i, n);
                        if (i != 0 && solid) {
                            *dst = *F_(c, c->fpost, cc, ib, n);
                        } else if (cut) {
                            double uT[3];
                            uT_of(c, c->tri[18 * n + ib - 1], uT);
                            double eu = EV[ib][0] * uT[0] + EV[ib][1] * uT[1] + EV[ib][2] * uT[2];
                            double rl = (c->flags & OR_REF_RHO) ? 1.0 : rw[cc];
                            double corr = 2.0 * WV[ib] * rl * eu / CS2;  /* Ladd term */
                            double fout = *F_(c, c->fpost, cc, ib, n);
                            *dst = fout - corr;
                            c->slink[18 * n + ib - 1] += 2.0 * fout - corr;
                        } else {
                            long s = nidx(c, wrap(sx, c->nx), wrap(sy, c->ny), wrap(sz, c->nz));
                            *dst = *F_(c, c->fpost, cc, i, s);
                        }
                    }
                }
            }
    /* momentum absorbed by the substrate (diagnostic): each bounce returns 2 f e_i */
    if (c->wall) {
        for (long n = 0; n < N; ++n) {
            int z = (int)(n / ((long)c->nx * c->ny));
            if (is_solid(c, z)) continue;
            for (int k = 1; k < NQ; ++k) {
                int z2 = z + EV[k][2];
                if (wrap(z2, c->nz) != 0) continue;
                for (int cc = 0; cc < 2; ++cc) {
                    double fo = *F_(c, c->fpost, cc, k, n);
                    for (int a = 0; a < 3; ++a) wallmom[a] += 2.0 * fo * EV[k][a];
                }
            }
        }
    }
    for (int a = 0; a < 3; ++a) c->mom_to_wall[a] += wallmom[a];
}

/* density interpolated for the far side of a cut (or wall) link: mean of the
 * node's own value and those of its neighbours reached through uncut fluid links */
static double rho_interp(const or_ctx *c, const double *rho, int x, int y, int z, long n) {
    if (c->flags & OR_MIRROR) return rho[n];
    double s = rho[n];
    int cnt = 1;
    for (int k = 1; k < NQ; ++k) {
        int z2 = z + EV[k][2];
        if (c->wall && wrap(z2, c->nz) == 0) continue;
        if (lmask(c, n) & (1u << (k - 1))) continue;
        long m = nidx(c, wrap(x + EV[k][0], c->nx), wrap(y + EV[k][1], c->ny), wrap(z2, c->nz));
        s += rho[m];
        ++cnt;
    }
    return s / cnt;
}

static void collide(or_ctx *c, double *Fsc_out) {
    long N = c->N;
    double *rho = c->rho;       /* [2][N] */
    double *psi = (double *)calloc(2 * N, sizeof(double));
    double *j = (double *)calloc(6 * N, sizeof(double));
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
        int z = (int)(n / ((long)c->nx * c->ny));
        for (int cc = 0; cc < 2; ++cc) {
            double r = 0, jx = 0, jy = 0, jz = 0;
            if (!is_solid(c, z))
                for (int i = 0; i < NQ; ++i) {
                    double f = *F_(c, c->fpre, cc, i, n);
                    r += f; jx += f * EV[i][0]; jy += f * EV[i][1]; jz += f * EV[i][2];
                }
            rho[cc * N + n] = r;
            j[(cc * 3 + 0) * N + n] = jx; j[(cc * 3 + 1) * N + n] = jy; j[(cc * 3 + 2) * N + n] = jz;
            psi[cc * N + n] = psi_of(r);
        }
    }
#pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < c->nz; ++z)
        for (int y = 0; y < c->ny; ++y)
            for (int x = 0; x < c->nx; ++x) {
                if (is_solid(c, z)) continue;
                long n = nidx(c, x, y, z);
                double Fc[2][3] = {{0, 0, 0}, {0, 0, 0}};
                double rho_far[2] = {-1.0, -1.0};
                for (int cc = 0; cc < 2; ++cc) {
                    int cb = 1 - cc;
                    double G = c->G;  /* G^{AB} = G^{BA} = G, G^{cc} = 0 */
                    for (int k = 1; k < NQ; ++k) {
                        int z2 = z + EV[k][2];
                        int wallk = c->wall && wrap(z2, c->nz) == 0;
                        int cutk = lmask(c, n) & (1u << (k - 1));
                        double pf;
                        if (wallk || cutk) {
                            if (rho_far[cb] < 0.0) rho_far[cb] = rho_interp(c, &rho[cb * N], x, y, z, n);
                            double r = rho_far[cb];
                            if (cutk && !wallk) {
                                /* wetting: the crossed element's capsule offsets the
                                 * interpolated densities, +wet for A and -wet for B */
                                int f;
                                const or_capsule *q = capsule_of(c, c->tri[18 * n + k - 1], &f);
                                r += cb == 0 ? q->wet : -q->wet;
                            }
                            pf = psi_of(r);
                            if (cutk && !wallk)  /* reaction on the crossed element */
                                c->slink[18 * n + k - 1] += psi[cc * N + n] * G * WV[k] * pf;
                        } else {
                            long m = nidx(c, wrap(x + EV[k][0], c->nx), wrap(y + EV[k][1], c->ny), wrap(z2, c->nz));
                            pf = psi[cb * N + m];
                        }
                        for (int a = 0; a < 3; ++a) Fc[cc][a] -= psi[cc * N + n] * G * WV[k] * pf * EV[k][a];
                    }
                }
                if (Fsc_out)
                    for (int cc = 0; cc < 2; ++cc)
                        for (int a = 0; a < 3; ++a) Fsc_out[(cc * 3 + a) * N + n] = Fc[cc][a];
                if (c->flags & OR_IBM) {  /* spread membrane force, shared by density */
                    double rt = rho[n] + rho[N + n];
                    for (int cc = 0; cc < 2; ++cc)
                        for (int a = 0; a < 3; ++a) Fc[cc][a] += c->fibm[a * N + n] * rho[cc * N + n] / rt;
                }
                /* velocity shift (Shan & Chen): common velocity weighted by 1/tau */
                double num[3] = {0, 0, 0}, den = 0.0;
                for (int cc = 0; cc < 2; ++cc) {
                    for (int a = 0; a < 3; ++a) num[a] += j[(cc * 3 + a) * N + n] / c->tau[cc];
                    den += rho[cc * N + n] / c->tau[cc];
                }
                double up[3] = {num[0] / den, num[1] / den, num[2] / den};
                double rt = rho[n] + rho[N + n];
                for (int a = 0; a < 3; ++a)
                    c->u[a * N + n] = (j[(0 * 3 + a) * N + n] + j[(1 * 3 + a) * N + n] + 0.5 * (Fc[0][a] + Fc[1][a])) / rt;
                for (int cc = 0; cc < 2; ++cc) {
                    double r = rho[cc * N + n];
                    double ueq[3];
                    for (int a = 0; a < 3; ++a) ueq[a] = up[a] + c->tau[cc] * Fc[cc][a] / r;
                    double feq[NQ];
                    equilibrium(r, ueq, feq);
                    for (int i = 0; i < NQ; ++i) {
                        double f = *F_(c, c->fpre, cc, i, n);
                        *F_(c, c->fpost, cc, i, n) = f - (f - feq[i]) / c->tau[cc];
                    }
                }
            }
    free(psi); free(j);
}

/* membrane forces of one capsule at its current positions (no coupling term) */
static void elastic_forces(const or_capsule *p, double *Fel, double *E3) {
    memset(Fel, 0, sizeof(double) * 3 * p->nv);
    double es = skalak(p->X, p->F, p->nf, p->refM, p->refA, p->refDet, p->kS, p->C, Fel);
    double eb = helfrich(p->X, p->F, p->nv, p->nf, p->kB, Fel);
    double ev = volume_penalty(p->X, p->F, p->nf, p->kV, p->V0, Fel);
    if (E3) { E3[0] = es; E3[1] = eb; E3[2] = ev; }
}

static void membrane_forces(or_ctx *c);
static void integrate(or_ctx *c);

static void membrane_update(or_ctx *c) {
    /* element momentum exchange of this step (links were recorded per node) */
    for (int ci = 0; ci < c->ncaps; ++ci) memset(c->caps[ci].FT_cur, 0, sizeof(double) * 3 * c->caps[ci].nf);
    double tot[3] = {0, 0, 0};
    for (long n = 0; n < c->N; ++n) {
        if (!c->mask[n]) continue;
        for (int k = 1; k < NQ; ++k) {
            if (!(c->mask[n] & (1u << (k - 1)))) continue;
            int f;
            or_capsule *p = capsule_of(c, c->tri[18 * n + k - 1], &f);
            double s = c->slink[18 * n + k - 1];
            for (int a = 0; a < 3; ++a) { p->FT_cur[3 * f + a] += s * EV[k][a]; tot[a] += s * EV[k][a]; }
        }
    }
    for (int a = 0; a < 3; ++a) c->mom_to_membrane[a] += tot[a];
    /* forces on nodes, all capsules at their current positions first */
    for (int ci = 0; ci < c->ncaps; ++ci) {
        or_capsule *p = &c->caps[ci];
        memset(p->Fcpl, 0, sizeof(double) * 3 * p->nv);
        for (int f = 0; f < p->nf; ++f) {
            for (int a = 0; a < 3; ++a) {
                double Fbar = 0.5 * (p->FT_cur[3 * f + a] + p->FT_prev[3 * f + a]);
                for (int v = 0; v < 3; ++v) p->Fcpl[3 * p->F[3 * f + v] + a] += Fbar / 3.0;
            }
        }
        memcpy(p->FT_prev, p->FT_cur, sizeof(double) * 3 * p->nf);
    }
    membrane_forces(c);
    integrate(c);
}

/* elastic (Fel) and Hertz (Fint) node forces of every capsule at the current
 * positions */
static void membrane_forces(or_ctx *c) {
    for (int ci = 0; ci < c->ncaps; ++ci) {
        or_capsule *p = &c->caps[ci];
        if (p->mode == 0) elastic_forces(p, p->Fel, NULL);
        else memset(p->Fel, 0, sizeof(double) * 3 * p->nv);
        memset(p->Fint, 0, sizeof(double) * 3 * p->nv);
        for (int v = 0; v < p->nv; ++v) {
            double d = p->X[3 * v + 2] - c->zrep;
            if (c->wall && d < c->delta0) p->Fint[3 * v + 2] += hertz_mag(c->xi, c->delta0, d);
        }
    }
    for (int ci = 0; ci < c->ncaps; ++ci)
        for (int cj = 0; cj < c->ncaps; ++cj) {
            if (ci == cj) continue;
            or_capsule *p = &c->caps[ci], *q = &c->caps[cj];
            for (int v = 0; v < p->nv; ++v)
                for (int w = 0; w < q->nv; ++w) {
                    double d3[3];
                    sub3(&p->X[3 * v], &q->X[3 * w], d3);
                    d3[0] -= c->nx * floor(d3[0] / c->nx + 0.5);  /* periodic images */
                    d3[1] -= c->ny * floor(d3[1] / c->ny + 0.5);
                    double d = norm3(d3);
                    if (d < c->delta0 && d > 0.0) {
                        double m = hertz_mag(c->xi, c->delta0, d);
                        for (int a = 0; a < 3; ++a) p->Fint[3 * v + a] += m * d3[a] / d;
                    }
                }
        }
}

/* node update (Eq. 9) and the per-capsule sums */
static void integrate(or_ctx *c) {
    for (int ci = 0; ci < c->ncaps; ++ci) {
        or_capsule *p = &c->caps[ci];
        double sF[3] = {0, 0, 0}, sT[3] = {0, 0, 0}, com[3] = {0, 0, 0}, sFt[3] = {0, 0, 0};
        for (int v = 0; v < p->nv; ++v)
            for (int a = 0; a < 3; ++a) com[a] += p->X[3 * v + a] / p->nv;
        for (int v = 0; v < p->nv; ++v) {
            double r[3], t[3];
            for (int a = 0; a < 3; ++a) {
                p->Ftot[3 * v + a] = p->Fel[3 * v + a] + p->Fint[3 * v + a] + p->Fcpl[3 * v + a];
                sF[a] += p->Fcpl[3 * v + a];
                sFt[a] += p->Ftot[3 * v + a];
                r[a] = p->X[3 * v + a] - com[a];
            }
            cross3(r, &p->Fcpl[3 * v], t);
            for (int a = 0; a < 3; ++a) sT[a] += t[a];
        }
        memcpy(p->force, sF, sizeof(sF));
        memcpy(p->torque, sT, sizeof(sT));
        /* area and volume of the mesh this step's forces were computed on */
        p->area = mesh_area(p->X, p->F, p->nf);
        p->volume = mesh_volume(p->X, p->F, p->nf);
        const int inertial = (c->flags & OR_INERTIAL) != 0;
        if (p->mode == 0) {          /* free: x += F/m, v = F/m (Eq. 9, dt = 1) */
            for (int k = 0; k < 3 * p->nv; ++k) {
                p->V[k] = (inertial ? p->V[k] : 0.0) + p->Ftot[k] / p->mass;
                p->X[k] += p->V[k];
            }
        } else if (p->mode == 1) {   /* frozen shape: rigid translation */
            double vr[3];
            for (int a = 0; a < 3; ++a) vr[a] = sFt[a] / (p->mass * p->nv);
            for (int v = 0; v < p->nv; ++v)
                for (int a = 0; a < 3; ++a) {
                    p->V[3 * v + a] = (inertial ? p->V[3 * v + a] : 0.0) + vr[a];
                    p->X[3 * v + a] += p->V[3 * v + a];
                }
        } else {                     /* fixed */
            memset(p->V, 0, sizeof(double) * 3 * p->nv);
        }
    }
}

/* Drying by species conversion.  The film is lowered by turning a mass dmA
 * of component A into component B each step, so the total mass stays put.
 * The nodes where A is the majority (rho^A > rho^B, this step's densities)
 * each give up the same fraction eps = dmA / (sum of their rho^A), at most 1,
 * of their post-collision A populations; the mass eps rho^A(x) a node gives
 * up joins its B populations in the rest-state proportions w_i.  The total A
 * inventory then falls by exactly dmA per step (by all of it once eps = 1). */
static void remove_mass(or_ctx *c) {
    const long N = c->N;
    double S = 0.0;
    for (long n = 0; n < N; ++n) {
        int z = (int)(n / ((long)c->nx * c->ny));
        if (!is_solid(c, z) && c->rho[n] > c->rho[N + n]) S += c->rho[n];
    }
    if (S <= 0.0) return;
    double eps = c->dmA / S;
    if (eps > 1.0) eps = 1.0;
    for (long n = 0; n < N; ++n) {
        int z = (int)(n / ((long)c->nx * c->ny));
        if (is_solid(c, z) || !(c->rho[n] > c->rho[N + n])) continue;
        const double dm = eps * c->rho[n];
        for (int i = 0; i < NQ; ++i) {
            *F_(c, c->fpost, 0, i, n) *= 1.0 - eps;
            if (!(c->flags & OR_REMOVE)) *F_(c, c->fpost, 1, i, n) += WV[i] * dm;
        }
    }
}

/* ------------------------------------------- diffuse-interface coupling */
/* Peskin's 4-point kernel: phi(r) = (3 - 2|r| + sqrt(1 + 4|r| - 4r^2)) / 8
 * for |r| <= 1, (5 - 2|r| - sqrt(-7 + 12|r| - 4r^2)) / 8 for 1 <= |r| <= 2,
 * 0 beyond; its shifts sum to 1 and have zero first moment at every offset */
static double peskin(double r) {
    r = fabs(r);
    if (r <= 1.0) return (3.0 - 2.0 * r + sqrt(1.0 + 4.0 * r - 4.0 * r * r)) / 8.0;
    if (r <= 2.0) return (5.0 - 2.0 * r - sqrt(-7.0 + 12.0 * r - 4.0 * r * r)) / 8.0;
    return 0.0;
}

/* the 64 lattice nodes around X (periodic) with their weights; solid
 * (substrate) nodes get index -1 */
static void ibm_stencil(const or_ctx *c, const double *X, long idx[64], double w[64]) {
    int b[3];
    double wa[3][4];
    for (int a = 0; a < 3; ++a) {
        b[a] = (int)floor(X[a]) - 1;
        for (int k = 0; k < 4; ++k) wa[a][k] = peskin(X[a] - (double)(b[a] + k));
    }
    int m = 0;
    for (int kz = 0; kz < 4; ++kz)
        for (int ky = 0; ky < 4; ++ky)
            for (int kx = 0; kx < 4; ++kx, ++m) {
                const int z = wrap(b[2] + kz, c->nz);
                w[m] = wa[0][kx] * wa[1][ky] * wa[2][kz];
                idx[m] = is_solid(c, z) ? -1 : nidx(c, wrap(b[0] + kx, c->nx), wrap(b[1] + ky, c->ny), z);
            }
}

/* f[3][N] += the force F at X spread with the kernel (nothing on solid nodes) */
static void ibm_spread_point(const or_ctx *c, const double *X, const double *F, double *f) {
    long idx[64];
    double w[64];
    ibm_stencil(c, X, idx, w);
    for (int m = 0; m < 64; ++m)
        if (idx[m] >= 0)
            for (int a = 0; a < 3; ++a) f[a * c->N + idx[m]] += F[a] * w[m];
}

/* the field u[3][N] interpolated at X (solid nodes carry zero velocity) */
static void ibm_interp_point(const or_ctx *c, const double *u, const double *X, double out[3]) {
    long idx[64];
    double w[64];
    ibm_stencil(c, X, idx, w);
    out[0] = out[1] = out[2] = 0.0;
    for (int m = 0; m < 64; ++m)
        if (idx[m] >= 0)
            for (int a = 0; a < 3; ++a) out[a] += u[a * c->N + idx[m]] * w[m];
}

/* membrane forces at the current positions, spread to the lattice */
static void ibm_spread(or_ctx *c) {
    memset(c->fibm, 0, sizeof(double) * 3 * c->N);
    for (int ci = 0; ci < c->ncaps; ++ci) memset(c->caps[ci].Fcpl, 0, sizeof(double) * 3 * c->caps[ci].nv);
    membrane_forces(c);
    for (int ci = 0; ci < c->ncaps; ++ci) {
        or_capsule *p = &c->caps[ci];
        for (int v = 0; v < p->nv; ++v) {
            double F[3];
            for (int a = 0; a < 3; ++a) F[a] = p->Fel[3 * v + a] + p->Fint[3 * v + a];
            ibm_spread_point(c, &p->X[3 * v], F, c->fibm);
        }
    }
}

/* nodes moved with the interpolated physical fluid velocity of this step;
 * force sums (the coupling force is zero: no link is cut), area, volume */
static void ibm_move(or_ctx *c) {
    for (int ci = 0; ci < c->ncaps; ++ci) {
        or_capsule *p = &c->caps[ci];
        for (int v = 0; v < p->nv; ++v)
            for (int a = 0; a < 3; ++a) p->Ftot[3 * v + a] = p->Fel[3 * v + a] + p->Fint[3 * v + a];
        memset(p->force, 0, sizeof(p->force));
        memset(p->torque, 0, sizeof(p->torque));
        p->area = mesh_area(p->X, p->F, p->nf);
        p->volume = mesh_volume(p->X, p->F, p->nf);
        if (p->mode != 0) { memset(p->V, 0, sizeof(double) * 3 * p->nv); continue; }
        for (int v = 0; v < p->nv; ++v) {
            double u[3];
            ibm_interp_point(c, c->u, &p->X[3 * v], u);
            for (int a = 0; a < 3; ++a) {
                p->V[3 * v + a] = u[a];
                p->X[3 * v + a] += u[a];
            }
        }
    }
}

double or_peskin(double r) { return peskin(r); }
void or_ibm_spread_point(const or_ctx *c, const double *X, const double *F, double *f) {
    ibm_spread_point(c, X, F, f);
}
void or_ibm_interp_point(const or_ctx *c, const double *u, const double *X, double *out) {
    ibm_interp_point(c, u, X, out);
}

void or_remove_mass(or_ctx *c, double dmA) { c->dmA = dmA; }

/* Alternative readings (OR_* flags above), 0 for the defaults. */
void or_set_flags(or_ctx *c, int flags) {
    c->flags = flags;
    if ((flags & OR_IBM) && !c->fibm) c->fibm = (double *)calloc(3 * (size_t)c->N, sizeof(double));
}

int or_step(or_ctx *c, int nsteps) {
    for (int s = 0; s < nsteps; ++s) {
        if (c->flags & OR_IBM) {
            stream(c);
            ibm_spread(c);
            collide(c, NULL);
            if (c->dmA > 0.0) remove_mass(c);
            ibm_move(c);
            /* the interior flags of the readouts follow the membrane */
            if (compute_cuts(c) != 0) return -1;
            compute_inside(c);
            c->step++;
            continue;
        }
        stream(c);
        collide(c, NULL);
        if (c->dmA > 0.0) remove_mass(c);
        membrane_update(c);
        int moving = 0;
        for (int ci = 0; ci < c->ncaps; ++ci) moving |= c->caps[ci].mode != 2;
        if (moving) {
            if (compute_cuts(c) != 0) return -1;
            compute_inside(c);
        }
        c->step++;
    }
    return 0;
}

/* ------------------------------------------------------------- readouts */
void or_fields(const or_ctx *c, double *rho, double *u) {
    if (rho) memcpy(rho, c->rho, sizeof(double) * 2 * c->N);
    if (u) memcpy(u, c->u, sizeof(double) * 3 * c->N);
}

void or_capsule_state(const or_ctx *c, int id, double *X, double *V, double *Fcpl,
                      double *Ftot, double out8[8]) {
    const or_capsule *p = &c->caps[id];
    if (X) memcpy(X, p->X, sizeof(double) * 3 * p->nv);
    if (V) memcpy(V, p->V, sizeof(double) * 3 * p->nv);
    if (Fcpl) memcpy(Fcpl, p->Fcpl, sizeof(double) * 3 * p->nv);
    if (Ftot) memcpy(Ftot, p->Ftot, sizeof(double) * 3 * p->nv);
    if (out8) {
        for (int a = 0; a < 3; ++a) { out8[a] = p->force[a]; out8[3 + a] = p->torque[a]; }
        out8[6] = p->area; out8[7] = p->volume;
    }
}

/* node velocities used by the moving-wall term of the next streaming (tests) */
void or_set_capsule_velocity(or_ctx *c, int id, const double *V) {
    memcpy(c->caps[id].V, V, sizeof(double) * 3 * c->caps[id].nv);
}

void or_momentum(const or_ctx *c, double fluid[3], double to_membrane[3], double to_wall[3]) {
    double m[3] = {0, 0, 0};
    for (int cc = 0; cc < 2; ++cc)
        for (int i = 0; i < NQ; ++i)
            for (long n = 0; n < c->N; ++n) {
                double f = c->fpost[((long)cc * NQ + i) * c->N + n];
                for (int a = 0; a < 3; ++a) m[a] += f * EV[i][a];
            }
    for (int a = 0; a < 3; ++a) {
        fluid[a] = m[a];
        to_membrane[a] = c->mom_to_membrane[a];
        to_wall[a] = c->mom_to_wall[a];
    }
}

void or_total_mass(const or_ctx *c, double m[2]) {
    for (int cc = 0; cc < 2; ++cc) {
        double s = 0.0;
        for (int i = 0; i < NQ; ++i)
            for (long n = 0; n < c->N; ++n) s += c->fpost[((long)cc * NQ + i) * c->N + n];
        m[cc] = s;
    }
}

void or_cuts(const or_ctx *c, uint32_t *mask, int *tri, uint8_t *inside) {
    if (mask) memcpy(mask, c->mask, sizeof(uint32_t) * c->N);
    if (tri) memcpy(tri, c->tri, sizeof(int) * 18 * c->N);
    if (inside) memcpy(inside, c->inside, c->N);
}

/* Film height per column (readout for the meniscus, Sec. 4.1): scanning up
 * from the substrate, the first change of phi = rhoA - rhoB from positive to
 * non-positive, linearly interpolated; NaN where that crossing touches a
 * capsule-interior node or no crossing exists. */
void or_meniscus_field(const or_ctx *c, const double *rho_in, double *h) {
    long N = c->N;
    const double *rho = rho_in ? rho_in : c->rho;
    for (int y = 0; y < c->ny; ++y)
        for (int x = 0; x < c->nx; ++x) {
            double out = NAN;
            for (int z = (c->wall ? 1 : 0); z + 1 < c->nz; ++z) {
                long n0 = nidx(c, x, y, z), n1 = nidx(c, x, y, z + 1);
                double p0 = rho[n0] - rho[N + n0], p1 = rho[n1] - rho[N + n1];
                if (p0 > 0.0 && p1 <= 0.0) {
                    if (!c->inside[n0] && !c->inside[n1]) out = z + p0 / (p0 - p1);
                    break;
                }
            }
            h[(long)y * c->nx + x] = out;
        }
}

/* ----------------------------------------------------- unit entry points */
void or_tables(int *e /*19*3*/, double *w /*19*/, int *op /*19*/) {
    init_weights();
    for (int i = 0; i < NQ; ++i) {
        for (int a = 0; a < 3; ++a) e[3 * i + a] = EV[i][a];
        w[i] = WV[i];
        op[i] = opp(i);
    }
}

void or_equilibrium(double rho, const double *u, double *feq) {
    init_weights();
    equilibrium(rho, u, feq);
}

/* Shan-Chen forces on the current post-collision densities of a context
 * without capsules (unit test of Eq. 10): F [2][3][N]. */
void or_sc_forces(or_ctx *c, double *F) {
    /* treat the post-collision populations as the streamed state */
    memcpy(c->fpre, c->fpost, sizeof(double) * 2 * NQ * c->N);
    double *save = (double *)malloc(sizeof(double) * 2 * NQ * c->N);
    memcpy(save, c->fpost, sizeof(double) * 2 * NQ * c->N);
    collide(c, F);
    memcpy(c->fpost, save, sizeof(double) * 2 * NQ * c->N);
    free(save);
}

/* Membrane energies [Skalak, Helfrich, volume] and elastic forces of a mesh
 * X with reference Xref (unit tests of Eqs. 6-8). */
void or_membrane(int nv, const double *X, const double *Xref, int nf, const int *F, double kS,
                 double C, double kB, double kV, double *E3, double *Fout, int which) {
    init_weights();
    double *refM = (double *)malloc(sizeof(double) * 3 * nf);
    double *refA = (double *)malloc(sizeof(double) * nf);
    double *refDet = (double *)malloc(sizeof(double) * nf);
    reference_state(Xref, F, nf, refM, refA, refDet);
    double V0 = mesh_volume(Xref, F, nf);
    if (Fout) memset(Fout, 0, sizeof(double) * 3 * nv);
    E3[0] = (which & 1) ? skalak(X, F, nf, refM, refA, refDet, kS, C, Fout) : 0.0;
    E3[1] = (which & 2) ? helfrich(X, F, nv, nf, kB, Fout) : 0.0;
    E3[2] = (which & 4) ? volume_penalty(X, F, nf, kV, V0, Fout) : 0.0;
    free(refM); free(refA); free(refDet);
}

double or_mesh_volume(const double *X, const int *F, int nf) { return mesh_volume(X, F, nf); }
double or_mesh_area(const double *X, const int *F, int nf) { return mesh_area(X, F, nf); }
double or_hertz(double xi, double delta0, double d) { return d < delta0 ? hertz_mag(xi, delta0, d) : 0.0; }

/* Brute force: every fluid lattice link of the box against every element of
 * every capsule (for tiny cases) -- same decision rule, no bounding boxes. */
void or_cuts_bruteforce(const or_ctx *c, uint32_t *mask, int *tri) {
    memset(mask, 0, sizeof(uint32_t) * c->N);
    for (long k = 0; k < 18 * c->N; ++k) tri[k] = -1;
    for (int z = 0; z < c->nz; ++z)
        for (int y = 0; y < c->ny; ++y)
            for (int x = 0; x < c->nx; ++x)
                for (int k = 1; k < NQ; ++k) {
                    if (!link_fluid(c, z, k)) continue;
                    long a = nidx(c, x, y, z);
                    for (int ci = 0; ci < c->ncaps; ++ci) {
                        const or_capsule *p = &c->caps[ci];
                        for (int f = 0; f < p->nf; ++f) {
                            double A[3], B[3], C[3];
                            tri_vertices_f(p, f, A, B, C);
                            /* nearest periodic image of the link to the element */
                            double cx = (A[0] + B[0] + C[0]) / 3.0, cy = (A[1] + B[1] + C[1]) / 3.0;
                            double px = x + c->nx * floor((cx - x) / c->nx + 0.5);
                            double py = y + c->ny * floor((cy - y) / c->ny + 0.5);
                            double P[3] = {px, py, z};
                            double Q[3] = {px + EV[k][0], py + EV[k][1], z + EV[k][2]};
                            if (seg_tri(P, Q, A, B, C)) {
                                int T = p->tri_base + f;
                                mask[a] ^= 1u << (k - 1);
                                if (tri[18 * a + k - 1] < 0 || T < tri[18 * a + k - 1]) tri[18 * a + k - 1] = T;
                            }
                        }
                    }
                }
}

/* ------------------------------------------- hooks for the oracle's pins */
/* Partner density across a cut or substrate link (reading c10) of component
 * `comp` at node (x, y, z), evaluated on the density field rho [N] given by
 * the caller and the context's current cut structure and substrate. */
double or_rho_interp(const or_ctx *c, const double *rho, int x, int y, int z) {
    init_weights();
    return rho_interp(c, rho, x, y, z, nidx(c, x, y, z));
}

/* Wetting of capsule id (Sec. 3.1, last paragraph: an offset added to the
 * interpolated densities tunes the contact angle; 0 is the neutral wetting
 * the paper uses).  Reading: on every link the capsule's membrane cuts, the
 * partner density interpolated for the Shan-Chen force is rho_interp + wet
 * for component A and rho_interp - wet for component B (the reaction on the
 * element uses the same values); substrate links stay neutral. */
void or_set_capsule_wetting(or_ctx *c, int id, double wet) { c->caps[id].wet = wet; }

/* Replace the context's cut structure (mask [N], elements [N*18]) and
 * recompute the interior flags from it. */
void or_set_cuts(or_ctx *c, const uint32_t *mask, const int *tri) {
    memcpy(c->mask, mask, sizeof(uint32_t) * c->N);
    memcpy(c->tri, tri, sizeof(int) * 18 * c->N);
    compute_inside(c);
}

/* Elastic (Eqs. 6-8) and interaction (Eq. 11) node forces [nv*3] of capsule
 * id from the last step (either may be NULL). */
void or_capsule_forces(const or_ctx *c, int id, double *Fel, double *Fint) {
    const or_capsule *p = &c->caps[id];
    if (Fel) memcpy(Fel, p->Fel, sizeof(double) * 3 * p->nv);
    if (Fint) memcpy(Fint, p->Fint, sizeof(double) * 3 * p->nv);
}

/* ------------------------------------------ meniscus profile and rise Z */
/* Meniscus profile around capsule id (Sec. 4.1 and reading c21) from a
 * column height field h [ny][nx] (NaN = no valid interface) and the xy
 * centroids cx, cy of all ncaps capsules:
 *  - h_inf: mean of the valid columns whose periodic distance to the nearest
 *    centroid is at least 0.9 times the largest such distance over the valid
 *    columns (the film far from every capsule);
 *  - rays: from the column nearest to capsule id's centroid along +x, -x, +y
 *    and -y; at distance r_k = k dr (k = 0 .. nr-1) the height is read by
 *    linear interpolation between the two columns that bracket r_k on the ray
 *    (periodic), a sample being invalid when either column is NaN;
 *  - zeta_k = (mean of the valid ray samples) - h_inf, NaN if none is valid;
 *  - Z = the largest valid zeta_k (the capillary rise), NaN if none.
 * r, zeta: [nr].  Returns h_inf. */
double or_meniscus_profile_of(const double *h, int nx, int ny, int ncaps, const double *cx,
                              const double *cy, int id, double dr, int nr, double *r,
                              double *zeta, double *Z) {
    double dmax = 0.0;
    double *dmin = (double *)malloc(sizeof(double) * (size_t)nx * ny);
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            double best = INFINITY;
            for (int k = 0; k < ncaps; ++k) {
                double dx = x - cx[k], dy = y - cy[k];
                dx -= nx * floor(dx / nx + 0.5);
                dy -= ny * floor(dy / ny + 0.5);
                double d = sqrt(dx * dx + dy * dy);
                if (d < best) best = d;
            }
            dmin[(long)y * nx + x] = best;
            if (!isnan(h[(long)y * nx + x]) && best > dmax) dmax = best;
        }
    double hs = 0.0;
    long hc = 0;
    for (long i = 0; i < (long)nx * ny; ++i)
        if (!isnan(h[i]) && dmin[i] >= 0.9 * dmax) { hs += h[i]; ++hc; }
    free(dmin);
    double hinf = hc ? hs / hc : NAN;
    int x0 = (int)lround(cx[id]), y0 = (int)lround(cy[id]);
    const int rx[4] = {1, -1, 0, 0}, ry[4] = {0, 0, 1, -1};
    double zmax = NAN;
    for (int k = 0; k < nr; ++k) {
        double rk = k * dr, s = 0.0;
        int cnt = 0;
        int j0 = (int)floor(rk);
        double t = rk - j0;
        for (int q = 0; q < 4; ++q) {
            int xa = wrap(x0 + rx[q] * j0, nx), ya = wrap(y0 + ry[q] * j0, ny);
            int xb = wrap(x0 + rx[q] * (j0 + 1), nx), yb = wrap(y0 + ry[q] * (j0 + 1), ny);
            double ha = h[(long)ya * nx + xa], hb = h[(long)yb * nx + xb];
            double v = (t == 0.0) ? ha : (1.0 - t) * ha + t * hb;
            if (!isnan(v)) { s += v; ++cnt; }
        }
        r[k] = rk;
        zeta[k] = cnt ? s / cnt - hinf : NAN;
        if (cnt && (isnan(zmax) || zeta[k] > zmax)) zmax = zeta[k];
    }
    if (Z) *Z = zmax;
    return hinf;
}

/* xy centroid of every capsule (mean of its node positions). */
static void centroids_xy(const or_ctx *c, double *cx, double *cy) {
    for (int k = 0; k < c->ncaps; ++k) {
        const or_capsule *p = &c->caps[k];
        double sx = 0.0, sy = 0.0;
        for (int v = 0; v < p->nv; ++v) { sx += p->X[3 * v]; sy += p->X[3 * v + 1]; }
        cx[k] = sx / p->nv;
        cy[k] = sy / p->nv;
    }
}

/* The profile of capsule id on the context's own height field (the
 * densities of the last step).  Returns h_inf. */
double or_meniscus_profile(const or_ctx *c, int id, double dr, int nr, double *r, double *zeta,
                           double *Z) {
    double *h = (double *)malloc(sizeof(double) * (size_t)c->nx * c->ny);
    double cx[MAXCAPS], cy[MAXCAPS];
    or_meniscus_field(c, NULL, h);
    centroids_xy(c, cx, cy);
    double hinf = or_meniscus_profile_of(h, c->nx, c->ny, c->ncaps, cx, cy, id, dr, nr, r, zeta, Z);
    free(h);
    return hinf;
}

/* ------------------------------------------------------- lateral force */
/* Lateral capillary force between capsules a and b (Eq. 3 sign convention,
 * reading c22): with e the unit xy vector from centroid a to centroid b
 * (nearest periodic image in x and y), F = 1/2 (F_b - F_a) . e, F_a and F_b
 * the fluid coupling forces on the capsules.  Negative = attraction.
 * Returns NaN when the centroids coincide in the xy plane. */
double or_lateral_force_of(const double *Fa, const double *Fb, const double *ca, const double *cb,
                           int nx, int ny) {
    double dx = cb[0] - ca[0], dy = cb[1] - ca[1];
    dx -= nx * floor(dx / nx + 0.5);
    dy -= ny * floor(dy / ny + 0.5);
    double L = sqrt(dx * dx + dy * dy);
    if (!(L > 0.0)) return NAN;
    return 0.5 * ((Fb[0] - Fa[0]) * dx + (Fb[1] - Fa[1]) * dy) / L;
}

/* The same for two capsules of the context (coupling forces of the last
 * step, centroids of the current node positions). */
double or_lateral_force(const or_ctx *c, int a, int b) {
    double cx[MAXCAPS], cy[MAXCAPS];
    centroids_xy(c, cx, cy);
    double ca[2] = {cx[a], cy[a]}, cb[2] = {cx[b], cy[b]};
    return or_lateral_force_of(c->caps[a].force, c->caps[b].force, ca, cb, c->nx, c->ny);
}

/* ------------------------------------------------- cut-structure override */
/* A crossing decision of link P->Q against element (A, B, C) is a near tie
 * when some perturbation of the inputs by at most `margin` lattice units can
 * flip it: each of the five orientation tests of seg_tri (the link ends
 * against the element plane, the link line against the three edges) is
 * classed +, - or undecided (|normalised value| < margin), and the decision
 * is ambiguous when an assignment of the undecided tests makes it a
 * crossing and another makes it none.  Plane tests are normalised to
 * distances by |n|, edge tests by |edge| |Q - P|. */
static int near_tie(const double *P, const double *Q, const double *A, const double *B,
                    const double *C, double margin) {
    double u[3], w[3], n[3], pq[3];
    sub3(B, A, u); sub3(C, A, w); cross3(u, w, n);
    sub3(Q, P, pq);
    double nn = norm3(n), lpq = norm3(pq);
    if (!(nn > 0.0)) return 1;
    double e1[3], e2[3], e3[3];
    sub3(B, A, e1); sub3(C, B, e2); sub3(A, C, e3);
    double v[5] = {orient3(A, B, C, P) / nn, orient3(A, B, C, Q) / nn,
                   orient3(P, Q, A, B) / (norm3(e1) * lpq), orient3(P, Q, B, C) / (norm3(e2) * lpq),
                   orient3(P, Q, C, A) / (norm3(e3) * lpq)};
    int cls[5];
    for (int k = 0; k < 5; ++k) cls[k] = fabs(v[k]) < margin ? 0 : (v[k] > 0.0 ? 1 : -1);
    /* can the two ends lie on different sides / on the same side? */
    int can_differ = cls[0] == 0 || cls[1] == 0 || cls[0] != cls[1];
    int can_same = cls[0] == 0 || cls[1] == 0 || cls[0] == cls[1];
    /* can the three edge tests agree / disagree? */
    int has_p = 0, has_m = 0, n_u = 0;
    for (int k = 2; k < 5; ++k) { has_p |= cls[k] == 1; has_m |= cls[k] == -1; n_u += cls[k] == 0; }
    int can_agree = !(has_p && has_m);
    int can_disagree = (has_p && has_m) || (n_u >= 1 && (has_p || has_m)) || n_u >= 2;
    int possible_true = can_differ && can_agree;
    int possible_false = can_same || can_disagree;
    return possible_true && possible_false;
}

/* Is any element's crossing decision for the link from node (x, y, z) along
 * e_k a near tie?  (Brute force over all elements, nearest periodic image of
 * the link to each element, single-precision node positions as in
 * compute_cuts.) */
static int link_near_tie(const or_ctx *c, int x, int y, int z, int k, double margin) {
    for (int ci = 0; ci < c->ncaps; ++ci) {
        const or_capsule *p = &c->caps[ci];
        for (int f = 0; f < p->nf; ++f) {
            double A[3], B[3], C[3];
            tri_vertices_f(p, f, A, B, C);
            double cx = (A[0] + B[0] + C[0]) / 3.0, cy = (A[1] + B[1] + C[1]) / 3.0;
            double cz = (A[2] + B[2] + C[2]) / 3.0;
            double px = x + c->nx * floor((cx - x) / c->nx + 0.5);
            double py = y + c->ny * floor((cy - y) / c->ny + 0.5);
            double pz = z + c->nz * floor((cz - z) / c->nz + 0.5);
            if (fabs(px - cx) > 18.0 || fabs(py - cy) > 18.0 || fabs(pz - cz) > 18.0) continue;
            double P[3] = {px, py, pz};
            double Q[3] = {px + EV[k][0], py + EV[k][1], pz + EV[k][2]};
            if (near_tie(P, Q, A, B, C, margin)) return 1;
        }
    }
    return 0;
}

/* Cut-list override (a diagnostic for free-membrane parity runs): compare a
 * cut structure computed elsewhere (mask [N], elements [N*18], e.g. by the
 * single-precision GPU path on its own node positions) with the oracle's.
 * Every link end where they differ (in the cut bit, or in the element of a
 * link both cut) must be a near tie of the oracle's own decision within
 * `margin`; then the given structure replaces the oracle's (interior flags
 * recomputed) and the number of differing link ends is returned (0: nothing
 * to do).  Otherwise nothing changes and the return value is minus the
 * number of differing link ends that are not near ties. */
long or_override_cuts(or_ctx *c, const uint32_t *mask, const int *tri, double margin) {
    long ndiff = 0, bad = 0;
    for (int z = 0; z < c->nz; ++z)
        for (int y = 0; y < c->ny; ++y)
            for (int x = 0; x < c->nx; ++x) {
                long n = nidx(c, x, y, z);
                uint32_t d = c->mask[n] ^ mask[n];
                for (int k = 1; k < NQ; ++k) {
                    uint32_t bit = 1u << (k - 1);
                    int differs = (d & bit) != 0;
                    if (!differs && (mask[n] & bit) && tri[18 * n + k - 1] != c->tri[18 * n + k - 1])
                        differs = 1;
                    if (!differs) continue;
                    ++ndiff;
                    if (!link_near_tie(c, x, y, z, k, margin)) ++bad;
                }
            }
    if (bad) return -bad;
    if (ndiff) or_set_cuts(c, mask, tri);
    return ndiff;
}

/* ------------------------------------------- theory of Sec. 2 (the check) */
/* Modified Bessel function of the second kind K_nu(x), x > 0, from the
 * integral representation K_nu(x) = int_0^inf exp(-x cosh t) cosh(nu t) dt
 * (a standard identity; the paper prints K_0 as a cosine integral and K_1 in
 * a garbled form, reading c5).  The integrand is analytic and decays
 * doubly exponentially, so the trapezoid rule with step 1/64 is exact to
 * rounding; the sum stops once a term falls below 1e-18 of the total. */
double or_bessel_k(int nu, double x) {
    if (!(x > 0.0)) return NAN;
    const double h = 1.0 / 64.0;
    double sum = 0.5 * exp(-x);  /* t = 0: cosh(0) = 1, halved (trapezoid end point) */
    for (int k = 1; k < 1000000; ++k) {
        double t = k * h;
        double term = exp(-x * cosh(t)) * cosh(nu * t);
        sum += term;
        if (term < 1e-18 * sum) break;
    }
    return sum * h;
}

/* Least-squares fit of the meniscus model zeta(r) = Q K_0(q r) (Eq. 12 with
 * Q = Gamma sin psi, Sec. 4.1) to the samples (r_k, zeta_k) with
 * rmin <= r_k <= rmax and a finite zeta_k: minimises
 * S(Q, q) = sum_k (zeta_k - Q K_0(q r_k))^2.  For a given q the best Q is
 * linear, Q(q) = sum zeta K_0 / sum K_0^2; S(Q(q), q) is scanned on 400
 * logarithmically spaced q in [1e-3, 3] and the best bracket refined by
 * golden-section search.  Returns the number of samples used (0: no fit);
 * rms = sqrt(S / samples). */
static double fit_S(const double *r, const double *z, int m, double q, double *Qout) {
    double zk = 0.0, kk = 0.0;
    for (int i = 0; i < m; ++i) {
        double k0 = or_bessel_k(0, q * r[i]);
        zk += z[i] * k0;
        kk += k0 * k0;
    }
    double Q = kk > 0.0 ? zk / kk : 0.0, S = 0.0;
    for (int i = 0; i < m; ++i) {
        double d = z[i] - Q * or_bessel_k(0, q * r[i]);
        S += d * d;
    }
    if (Qout) *Qout = Q;
    return S;
}

int or_meniscus_fit(const double *r, const double *zeta, int n, double rmin, double rmax, double *Q,
                    double *q, double *rms) {
    double *rr = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
    double *zz = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
    int m = 0;
    for (int i = 0; i < n; ++i)
        if (r[i] >= rmin && r[i] <= rmax && isfinite(zeta[i]) && r[i] > 0.0) { rr[m] = r[i]; zz[m] = zeta[i]; ++m; }
    if (m < 2) { free(rr); free(zz); *Q = *q = *rms = NAN; return 0; }
    const int NS = 400;
    const double lq0 = log(1e-3), lq1 = log(3.0);
    int best = 0;
    double bestS = INFINITY;
    for (int i = 0; i < NS; ++i) {
        double S = fit_S(rr, zz, m, exp(lq0 + (lq1 - lq0) * i / (NS - 1)), NULL);
        if (S < bestS) { bestS = S; best = i; }
    }
    double a = lq0 + (lq1 - lq0) * (best > 0 ? best - 1 : 0) / (NS - 1);
    double b = lq0 + (lq1 - lq0) * (best < NS - 1 ? best + 1 : NS - 1) / (NS - 1);
    const double g = (sqrt(5.0) - 1.0) / 2.0;
    double c = b - g * (b - a), d = a + g * (b - a);
    double Sc = fit_S(rr, zz, m, exp(c), NULL), Sd = fit_S(rr, zz, m, exp(d), NULL);
    for (int it = 0; it < 200 && b - a > 1e-15; ++it) {
        if (Sc < Sd) { b = d; d = c; Sd = Sc; c = b - g * (b - a); Sc = fit_S(rr, zz, m, exp(c), NULL); }
        else { a = c; c = d; Sc = Sd; d = a + g * (b - a); Sd = fit_S(rr, zz, m, exp(d), NULL); }
    }
    *q = exp(0.5 * (a + b));
    double S = fit_S(rr, zz, m, *q, Q);
    *rms = sqrt(S / m);
    free(rr); free(zz);
    return m;
}

/* Lateral capillary force between two particles of capillary charges Q1, Q2
 * at centre distance L (Eq. 13): F = -2 pi q gamma Q1 Q2 K_1(q L); negative is
 * attraction. */
double or_capillary_force(double q, double gamma, double Q1, double Q2, double L) {
    const double pi = 3.14159265358979323846;
    return -2.0 * pi * q * gamma * Q1 * Q2 * or_bessel_k(1, q * L);
}
