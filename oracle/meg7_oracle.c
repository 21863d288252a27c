/*
 * Plain FP64 CPU oracle of the MEG7-prim residual and its TVD-RK3 time step
 * (Chamarthi, "Efficient high-order gradient-based reconstruction for
 * compressible flows", arXiv:2305.00762).
 *
 * TEST INFRASTRUCTURE ONLY. This file exists so that tests can check the CUDA
 * path against an independent, slow and obviously correct restatement of the
 * paper. Only tests/, __graft_entry__.smoke() and the cpu_baseline /
 * reference leg of bench.py may load the library built from it. The CUDA path
 * never calls it, and the two share no source, header, table or helper.
 *
 * Every step follows the paper's order and notation, written as plain loops.
 * It is compiled with -ffp-contract=off so every a*b+c rounds twice, in the
 * order written here. OpenMP (when available) only splits independent rows
 * between threads; the arithmetic of each face and cell does not change.
 *
 * Readings of points the paper leaves open (each one is listed in the design
 * notes of the repository):
 *  R1  dimension-by-dimension (Sec. 2.1): x- and y-face fluxes are computed from
 *      the same stage state and their differences summed (Eq. deriv).
 *  R2  characteristic projection (Sec. 2.3, last paragraph): at face j+1/2 the
 *      primitive x-Jacobian is frozen at the arithmetic mean of U_j and
 *      U_{j+1}; U and U' of every stencil cell are projected with its left
 *      eigenvectors, each characteristic field is reconstructed, and the result
 *      is mapped back with the right eigenvectors. y faces swap u and v.
 *  R3  the MP test and limiter run at every face, whatever sigma is; Q_L, Q_R
 *      always come from MEG7 (Sec. 2.4, "computed independently").
 *  R4  detector regularisation: psi = (2ab + eps)/(a^2 + b^2 + eps) with the
 *      printed eps = 0.9 psi_c xi^2 / (1 - 0.9 psi_c), xi = 1e-3 (Eq. buffer);
 *      the printed ratio 2/(a/b + b/a) is undefined for a = 0 or b = 0.
 *  R5  xi = 7 in the MP bound (Eq. alpha); the hat on Phi_{j-1} in the LC bound
 *      and the index i in Eq. mp-procedure / flux-right are read as plain j.
 *  R6  the right-side MP value at j+1/2 is the left formula mirrored about the
 *      face: cell j+1-k plays cell j+k and Phi' changes sign (this mirror
 *      turns Eq. grb's left formula into its printed right formula).
 *  R7  HLLC (Toro 1994) written as 1/2(F_L+F_R) - 1/2|A|(Q_R-Q_L) (Eq.
 *      Riemann_revisit): |A| dQ = |S_L|(Q*_L-Q_L) + |S*|(Q*_R-Q*_L)
 *      + |S_R|(Q_R-Q*_R), wave speeds S_L = min(u_L-c_L, u~-c~),
 *      S_R = max(u_R+c_R, u~+c~) from Roe averages (Einfeldt bounds).
 *  R8  viscous faces (Sec. 2.1, 1D form extended dimension by dimension):
 *      normal derivatives of u, v and T by alpha-damping (Eq. alphad,
 *      alpha_v = 4); tangential derivatives the mean of the two cell-centre
 *      sixth-order values; face velocities the arithmetic mean; T = gamma p/rho
 *      (Eq. visc with Cp = 1/(gamma-1)); T' by the chain rule from the shared
 *      rho', p'; heat conductivity mu/(Pr (gamma-1)) (Eq. visc-interface).
 *  R9  G = 6 ghost layers: the LC bound at j+1/2 uses d_{j-1}, which uses
 *      Phi'_{j-2}, which uses Phi_{j-5}.
 *  R22 positivity fallback: a reconstructed face state with rho <= 0 or
 *      p <= 0 is replaced by the state of the cell on its side of the face
 *      (first order there); the paper prints no such rule, but the double
 *      Mach reflection (Example 8) reconstructs a negative pressure at the
 *      shock's foot in its first step without it. States that stay positive
 *      are untouched.
 *  R24 shock-stable HLLC (Examples 7 and 8 cite Fleischmann, Adami and Adams
 *      2020 without restating it): the HLLC-LM flux of that work, in the
 *      |A| form of R7. The acoustic terms |S_L|(Q*_L-Q_L) and |S_R|(Q_R-Q*_R)
 *      are scaled by phi = sin(pi/2 min(1, Ma/Ma_lim)), Ma = max(|u_L|/c_L,
 *      |u_R|/c_R) with the face-normal velocities, Ma_lim = 0.1; S_L, S_R,
 *      S* and the star states are those of R7. phi = 1 (Ma >= Ma_lim, every
 *      supersonic face) gives R7 exactly.
 *  R23 time-dependent boundaries: the RK stages of a step from t with step
 *      dt see the boundary at t, t + dt and t + dt/2 (Eq. rk's stage times).
 *  R20 MEG7-cons (Sec. 2.2, conservative reconstruction): Q and its
 *      sixth-order gradients are projected with the left eigenvectors of the
 *      conservative flux Jacobian frozen at the same mean state as in R2
 *      (H = c^2/(gamma-1) + (u^2+v^2)/2); the viscous terms take u', v' from
 *      the chain rule printed in Sec. 2.2 and T' = gamma (p'/rho - p rho'/rho^2)
 *      with p' = (gamma-1)(E' - u (rho u)' - v (rho v)' + (u^2+v^2) rho'/2).
 */
#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>

#define OR_G 6 /* ghost layers, reading R9 */

enum {
    OR_BC_PERIODIC = 0,
    OR_BC_TRANSMISSIVE = 1,
    OR_BC_NOSLIP_WALL = 2,
    OR_BC_SYMMETRY = 3,
    OR_BC_CUSTOM = 4, /* described by or_cfg.side[] */
    OR_BC_FIXED = 5   /* inside a side description: a fixed primitive state */
};

/* A custom side (the double Mach reflection of Woodward and Colella,
 * Example 8, needs them): the ghost cells beside interior cell k of the side
 * (centre at (k + 1/2) h along it) take kind_lo when that centre lies below
 * s0 + speed * t, else kind_hi; OR_BC_FIXED holds the primitive state lo or
 * hi. */
typedef struct {
    int kind_lo, kind_hi;
    double s0, speed;
    double lo[4], hi[4];
} or_side;
enum { OR_OK = 0, OR_ERR_ARG = -1, OR_ERR_NONPHYSICAL = -3, OR_ERR_NOMEM = -7 };

typedef struct {
    int nx, ny;               /* interior cells in x and y */
    double dx, dy;            /* cell sizes */
    double gamma, mu, Pr;     /* ratio of specific heats, viscosity, Prandtl */
    int bc[4];                /* west, east, south, north (OR_BC_*) */
    int order;                /* 7 = MEG7 (Eq. grb / flux-full); 4 = alpha=4, beta=0 subset */
    int cons;                 /* 0 = MEG7-prim (reconstruct U), 1 = MEG7-cons (reconstruct Q) */
    double t;                 /* time of the state (custom sides may move with it) */
    or_side side[4];          /* descriptions of OR_BC_CUSTOM sides */
    int riemann;              /* 0 = HLLC (R7), 1 = shock-stable HLLC-LM (R24) */
} or_cfg;

#define OR_MA_LIMIT 0.1               /* Ma_lim of reading R24 */
#define OR_HALF_PI 1.5707963267948966 /* pi / 2 rounded to double */

/* ---------------------------------------------------------------------- */
/* Scalar building blocks, each one equation of the paper.                 */
/* ---------------------------------------------------------------------- */

static double sgn(double a) { return (a > 0.0) ? 1.0 : ((a < 0.0) ? -1.0 : 0.0); }

/* Eq. alpha: minmod(a,b) = 1/2 (sign(a) + sign(b)) min(|a|,|b|). */
static double minmod(double a, double b) { return 0.5 * (sgn(a) + sgn(b)) * fmin(fabs(a), fabs(b)); }

static double min3(double a, double b, double c) { return fmin(a, fmin(b, c)); }
static double max3(double a, double b, double c) { return fmax(a, fmax(b, c)); }

/* Eq. six (= Eq. sixth-ordergrad times dx): the dx-scaled sixth-order explicit
 * gradient Phi'_j = dx (dPhi/dx)_j from phi[0..6] = Phi_{j-3..j+3}. */
double or_grad6(const double *phi)
{
    return (45.0 * (phi[4] - phi[2]) - 9.0 * (phi[5] - phi[1]) + (phi[6] - phi[0])) / 60.0;
}

/* Eq. grb, left value at j+1/2 from phi[0..4] = Phi_{j-2..j+2} and
 * dphi[0..4] = Phi'_{j-2..j+2} (only j-1..j+1 enter). */
double or_grb_left(const double *phi, const double *dphi)
{
    return (420.0 * dphi[2] + 60.0 * dphi[1] - 60.0 * dphi[3] + 478.0 * phi[2] + 178.0 * phi[1]
            + 3.0 * phi[0] + 178.0 * phi[3] + 3.0 * phi[4]) / 840.0;
}

/* Eq. grb, right value at j+1/2 from phi[0..4] = Phi_{j-1..j+3} and
 * dphi[0..4] = Phi'_{j-1..j+3} (only j..j+2 enter). */
double or_grb_right(const double *phi, const double *dphi)
{
    return (60.0 * dphi[1] - 420.0 * dphi[2] - 60.0 * dphi[3] + 178.0 * phi[1] + 3.0 * phi[0]
            + 478.0 * phi[2] + 178.0 * phi[3] + 3.0 * phi[4]) / 840.0;
}

/* Remark after Eq. grb (Sec. 2.2) and Sec. 3 "Comparison between fourth-order
 * and seventh-order": the alpha = 4, beta = 0 member of the family. Written
 * from Eqs. lingrb, how-second, good_6tth-order_scheme_flux and alpha-beta:
 * Phi^L = Phi_j + Phi'_j/2 + Phi''_j/12 with
 * Phi''_j = (Phi'_{j+1/2} - Phi'_{j-1/2}) (dx-scaled), and
 * Phi'_{j+1/2} = 1/2(Phi'_j + Phi'_{j+1}) + alpha/2 (Phi_R - Phi_L),
 * Phi_L = Phi_j + Phi'_j/2 + beta (Phi_{j+1} - 2 Phi_j + Phi_{j-1}),
 * Phi_R = Phi_{j+1} - Phi'_{j+1}/2 + beta (Phi_{j+2} - 2 Phi_{j+1} + Phi_j). */
static double alphabeta_face_grad(const double *phi, const double *dphi, int j, double alpha, double beta)
{
    /* face between array cells j and j+1 */
    double pl = phi[j] + 0.5 * dphi[j] + beta * (phi[j + 1] - 2.0 * phi[j] + phi[j - 1]);
    double pr = phi[j + 1] - 0.5 * dphi[j + 1] + beta * (phi[j + 2] - 2.0 * phi[j + 1] + phi[j]);
    return 0.5 * (dphi[j] + dphi[j + 1]) + 0.5 * alpha * (pr - pl);
}

/* Left value at j+1/2 of the (alpha, beta) family from Phi_{j-2..j+2} and
 * Phi'_{j-2..j+2}: Eq. lingrb with the second derivative of Eq. how-second. */
double or_grb_alphabeta_left(const double *phi, const double *dphi, double alpha, double beta)
{
    /* array index 2 is cell j */
    double gp = alphabeta_face_grad(phi, dphi, 2, alpha, beta);  /* j+1/2 */
    double gm = alphabeta_face_grad(phi, dphi, 1, alpha, beta);  /* j-1/2 */
    double d2 = gp - gm;                                         /* dx^2 Phi''_j */
    return phi[2] + 0.5 * dphi[2] + d2 / 12.0;
}

/* Left value of the scheme of order `order` (7: Eq. grb; 4: alpha=4, beta=0). */
static double grb_left(int order, const double *phi, const double *dphi)
{
    if (order == 4)
        return or_grb_alphabeta_left(phi, dphi, 4.0, 0.0);
    return or_grb_left(phi, dphi);
}

/* Eqs. mp5Condition, alpha and mp-procedure: the MEG7 left value at j+1/2.
 * phi[0..4] = Phi_{j-2..j+2}, dphi[0..4] = Phi'_{j-2..j+2}. */
static double meg_left(int order, const double *phi, const double *dphi)
{
    const double xi = 7.0; /* Eq. alpha, reading R5 */
    double pl = grb_left(order, phi, dphi);
    double pj = phi[2];
    double pmp = pj + minmod(phi[3] - pj, xi * (pj - phi[1]));
    if ((pl - pj) * (pl - pmp) <= 1e-40)
        return pl;
    /* d_k = 2(Phi_{k+1} - 2Phi_k + Phi_{k-1}) - 0.5(Phi'_{k+1} - Phi'_{k-1}) */
    double dm1 = 2.0 * (phi[2] - 2.0 * phi[1] + phi[0]) - 0.5 * (dphi[2] - dphi[0]); /* d_{j-1} */
    double d0 = 2.0 * (phi[3] - 2.0 * phi[2] + phi[1]) - 0.5 * (dphi[3] - dphi[1]);  /* d_j   */
    double dp1 = 2.0 * (phi[4] - 2.0 * phi[3] + phi[2]) - 0.5 * (dphi[4] - dphi[2]); /* d_{j+1} */
    double md = 0.5 * (pj + phi[3]) - 0.5 * minmod(d0, dp1);
    double ul = pj + xi * (pj - phi[1]);
    double lc = 0.5 * (3.0 * pj - phi[1]) + (4.0 / 3.0) * minmod(d0, dm1);
    double pmin = fmax(min3(pj, phi[3], md), min3(pj, ul, lc));
    double pmax = fmin(max3(pj, phi[3], md), max3(pj, ul, lc));
    return pl + minmod(pmin - pl, pmax - pl);
}

/* MEG7 left value (exported for tests). */
double or_meg7_left(const double *phi, const double *dphi) { return meg_left(7, phi, dphi); }

/* MEG7 right value at j+1/2 from phi[0..4] = Phi_{j-1..j+3} and
 * dphi[0..4] = Phi'_{j-1..j+3}: reading R6, the left procedure applied to the
 * mirrored stencil (cell j+1-k plays cell j+k, Phi' changes sign). */
static double meg_right(int order, const double *phi, const double *dphi)
{
    double mphi[5], mdphi[5];
    for (int k = 0; k < 5; ++k) {
        mphi[k] = phi[4 - k];
        mdphi[k] = -dphi[4 - k];
    }
    return meg_left(order, mphi, mdphi);
}

double or_meg7_right(const double *phi, const double *dphi) { return meg_right(7, phi, dphi); }

/* Eq. flux-full: F(f_L) at j+1/2 from f[0..8] = f_{j-4..j+4}. */
double or_flux_recon_left(const double *f)
{
    return (568.0 * f[4] - 146.0 * f[3] + 22.0 * f[2] + 2.0 * f[1] - f[0] + 484.0 * f[5] - 104.0 * f[6]
            + 16.0 * f[7] - f[8]) / 840.0;
}

/* Eq. flux-right: F(f_R) at j+1/2 from f[0..8] = f_{j-3..j+5}. */
double or_flux_recon_right(const double *f)
{
    return (-f[8] + 2.0 * f[7] + 22.0 * f[6] - 146.0 * f[5] + 568.0 * f[4] + 484.0 * f[3] - 104.0 * f[2]
            + 16.0 * f[1] - f[0]) / 840.0;
}

/* Sec. 3 "Comparison between fourth-order and seventh-order", Eq. fourth:
 * the alpha = 4, beta = 0 flux reconstruction, f[0..8] = f_{j-4..j+4}. */
double or_flux_recon4_left(const double *f)
{
    return (1050.0 * f[4] - 309.0 * f[3] + 64.0 * f[2] - 3.0 * f[1] - f[0] + 771.0 * f[5] - 152.0 * f[6]
            + 21.0 * f[7] - f[8]) / 1440.0;
}

static double flux_recon_left(int order, const double *f)
{
    return (order == 4) ? or_flux_recon4_left(f) : or_flux_recon_left(f);
}

/* Right flux reconstruction: the left one mirrored about the face (the same
 * mirror maps Eq. flux-full onto Eq. flux-right). f[0..8] = f_{j-3..j+5}. */
static double flux_recon_right(int order, const double *f)
{
    if (order != 4)
        return or_flux_recon_right(f);
    double m[9];
    for (int k = 0; k < 9; ++k)
        m[k] = f[8 - k];
    return or_flux_recon4_left(m);
}

/* Eq. detector and the line before it, with reading R4: psi_j from
 * rho[0..4] = rho_{j-2..j+2}. */
double or_psi(const double *rho)
{
    const double psi_c = 0.5, xi = 1e-3;
    const double eps = 0.9 * psi_c / (1.0 - 0.9 * psi_c) * xi * xi;
    double a = fabs(rho[2] - rho[1]) + fabs(rho[2] - 2.0 * rho[1] + rho[0]);
    double b = fabs(rho[2] - rho[3]) + fabs(rho[2] - 2.0 * rho[3] + rho[4]);
    return (2.0 * a * b + eps) / (a * a + b * b + eps);
}

/* Eq. pressure: conservative (rho, rho u, rho v, E) -> primitive (rho, u, v, p). */
static void cons_to_prim(double gamma, const double *q, double *w)
{
    double rho = q[0];
    double u = q[1] / rho;
    double v = q[2] / rho;
    w[0] = rho;
    w[1] = u;
    w[2] = v;
    w[3] = (gamma - 1.0) * (q[3] - rho * (u * u + v * v) / 2.0);
}

/* Sec. 1: E = p/(gamma-1) + rho (u^2 + v^2)/2 for primitive (rho, un, ut, p). */
static void prim_to_cons(double gamma, const double *w, double *q)
{
    q[0] = w[0];
    q[1] = w[0] * w[1];
    q[2] = w[0] * w[2];
    q[3] = w[3] / (gamma - 1.0) + w[0] * (w[1] * w[1] + w[2] * w[2]) / 2.0;
}

/* Sec. 1, F^c for primitive (rho, un, ut, p) in the face-normal frame:
 * (rho un, rho un^2 + p, rho un ut, un (E + p)); the 2D form drops the w rows. */
static void euler_flux(double gamma, const double *w, double *f)
{
    double q[4];
    prim_to_cons(gamma, w, q);
    f[0] = w[0] * w[1];
    f[1] = w[0] * w[1] * w[1] + w[3];
    f[2] = w[0] * w[1] * w[2];
    f[3] = w[1] * (q[3] + w[3]);
}

/* Eq. Riemann_revisit with HLLC (reading R7), or with the HLLC-LM flux of
 * reading R24 if lm != 0. WL, WR: primitive left/right face states
 * (rho, un, ut, p); FL, FR: the face fluxes that enter the central part
 * (hybrid F^c_L, F^c_R). Writes the numerical flux Fh. */
static void hllc_face(double gamma, int lm, const double *WL, const double *WR, const double *FL, const double *FR,
                      double *Fh)
{
    double QL[4], QR[4];
    prim_to_cons(gamma, WL, QL);
    prim_to_cons(gamma, WR, QR);
    double rL = WL[0], uL = WL[1], vL = WL[2], pL = WL[3];
    double rR = WR[0], uR = WR[1], vR = WR[2], pR = WR[3];
    double cL = sqrt(gamma * pL / rL), cR = sqrt(gamma * pR / rR);
    double HL = (QL[3] + pL) / rL, HR = (QR[3] + pR) / rR;
    /* Roe averages */
    double sL = sqrt(rL), sR = sqrt(rR);
    double ut = (sL * uL + sR * uR) / (sL + sR);
    double vt = (sL * vL + sR * vR) / (sL + sR);
    double Ht = (sL * HL + sR * HR) / (sL + sR);
    double ct = sqrt((gamma - 1.0) * (Ht - (ut * ut + vt * vt) / 2.0));
    double SL = fmin(uL - cL, ut - ct);
    double SR = fmax(uR + cR, ut + ct);
    double Ss = (pR - pL + rL * uL * (SL - uL) - rR * uR * (SR - uR)) / (rL * (SL - uL) - rR * (SR - uR));
    /* HLLC star states (Toro 1994) */
    double QsL[4], QsR[4];
    double kL = rL * (SL - uL) / (SL - Ss);
    double kR = rR * (SR - uR) / (SR - Ss);
    QsL[0] = kL;
    QsL[1] = kL * Ss;
    QsL[2] = kL * vL;
    QsL[3] = kL * (QL[3] / rL + (Ss - uL) * (Ss + pL / (rL * (SL - uL))));
    QsR[0] = kR;
    QsR[1] = kR * Ss;
    QsR[2] = kR * vR;
    QsR[3] = kR * (QR[3] / rR + (Ss - uR) * (Ss + pR / (rR * (SR - uR))));
    /* reading R24: the acoustic wave speeds of the dissipation scaled by phi */
    double aL = fabs(SL), aR = fabs(SR);
    if (lm) {
        double Ma = fmax(fabs(uL) / cL, fabs(uR) / cR);
        double z = fmin(1.0, Ma / OR_MA_LIMIT);
        double phi = z < 1.0 ? sin(OR_HALF_PI * z) : 1.0;
        aL *= phi;
        aR *= phi;
    }
    for (int m = 0; m < 4; ++m) {
        double adq = aL * (QsL[m] - QL[m]) + fabs(Ss) * (QsR[m] - QsL[m]) + aR * (QR[m] - QsR[m]);
        Fh[m] = 0.5 * (FL[m] + FR[m]) - 0.5 * adq;
    }
}

void or_hllc(double gamma, const double *WL, const double *WR, const double *FL, const double *FR, double *Fh)
{
    hllc_face(gamma, 0, WL, WR, FL, FR, Fh);
}

void or_hllc_lm(double gamma, const double *WL, const double *WR, const double *FL, const double *FR, double *Fh)
{
    hllc_face(gamma, 1, WL, WR, FL, FR, Fh);
}

/* ---------------------------------------------------------------------- */
/* Padded grids: (nx + 2G) x (ny + 2G) cells, x fastest, cell (j, i) of the */
/* interior at index (i + G) * W + (j + G).                                 */
/* ---------------------------------------------------------------------- */

static ptrdiff_t pidx(const or_cfg *c, int j, int i) { return (ptrdiff_t)(i + OR_G) * (c->nx + 2 * OR_G) + (j + OR_G); }

/* Source cell of ghost coordinate k along an axis of n interior cells with the
 * low/high boundary conditions; *flip = 1 if the velocity components named by
 * the condition change sign. Periodic wraps; transmissive copies the nearest
 * interior cell; a no-slip wall and a symmetry plane mirror about the face. */
static int ghost_source(int k, int n, int bc_lo, int bc_hi, int *flip_normal, int *flip_tangential)
{
    *flip_normal = 0;
    *flip_tangential = 0;
    if (k >= 0 && k < n)
        return k;
    int bc = (k < 0) ? bc_lo : bc_hi;
    switch (bc) {
    case OR_BC_PERIODIC:
        return ((k % n) + n) % n;
    case OR_BC_TRANSMISSIVE:
        return (k < 0) ? 0 : n - 1;
    case OR_BC_NOSLIP_WALL:
        *flip_normal = 1;
        *flip_tangential = 1;
        return (k < 0) ? -1 - k : 2 * n - 1 - k;
    default: /* OR_BC_SYMMETRY */
        *flip_normal = 1;
        return (k < 0) ? -1 - k : 2 * n - 1 - k;
    }
}

/* Ghost-cell boundary conditions (Sec. 3, ghost cell approach): first the x
 * ghosts of the interior rows, then the y ghosts of every column, so corner
 * ghosts take the y image of the x ghosts. Qp: 4 padded planes. */
/* Kind of side `sd` beside the cell with tangential index k (centre at
 * (k + 1/2) h) at time t; a fixed state is returned as a conservative vector
 * in q. Non-custom sides return their own kind. */
static int side_kind(const or_cfg *c, int sd, int k, double h, double q[4])
{
    if (c->bc[sd] != OR_BC_CUSTOM)
        return c->bc[sd];
    const or_side *S = &c->side[sd];
    int lo = (k + 0.5) * h < S->s0 + S->speed * c->t;
    int kind = lo ? S->kind_lo : S->kind_hi;
    if (kind == OR_BC_FIXED) {
        const double *w = lo ? S->lo : S->hi;
        q[0] = w[0];
        q[1] = w[0] * w[1];
        q[2] = w[0] * w[2];
        q[3] = w[3] / (c->gamma - 1.0) + 0.5 * w[0] * (w[1] * w[1] + w[2] * w[2]);
    }
    return kind;
}

void or_fill_ghosts(const or_cfg *c, double *Qp)
{
    const int nx = c->nx, ny = c->ny;
    const ptrdiff_t N = (ptrdiff_t)(nx + 2 * OR_G) * (ny + 2 * OR_G);
    for (int i = 0; i < ny; ++i) {
        for (int j = -OR_G; j < nx + OR_G; ++j) {
            if (j >= 0 && j < nx)
                continue;
            int fn, ft;
            double fixed[4];
            int kind = side_kind(c, j < 0 ? 0 : 1, i, c->dy, fixed);
            ptrdiff_t d = pidx(c, j, i);
            if (kind == OR_BC_FIXED) {
                for (int m = 0; m < 4; ++m)
                    Qp[m * N + d] = fixed[m];
                continue;
            }
            int s = ghost_source(j, nx, j < 0 ? kind : c->bc[0], j < 0 ? c->bc[1] : kind, &fn, &ft);
            ptrdiff_t o = pidx(c, s, i);
            Qp[0 * N + d] = Qp[0 * N + o];
            Qp[1 * N + d] = fn ? -Qp[1 * N + o] : Qp[1 * N + o]; /* x momentum is normal */
            Qp[2 * N + d] = ft ? -Qp[2 * N + o] : Qp[2 * N + o];
            Qp[3 * N + d] = Qp[3 * N + o];
        }
    }
    for (int i = -OR_G; i < ny + OR_G; ++i) {
        if (i >= 0 && i < ny)
            continue;
        for (int j = -OR_G; j < nx + OR_G; ++j) {
            int fn, ft;
            double fixed[4];
            int kind = side_kind(c, i < 0 ? 2 : 3, j, c->dx, fixed);
            ptrdiff_t d = pidx(c, j, i);
            if (kind == OR_BC_FIXED) {
                for (int m = 0; m < 4; ++m)
                    Qp[m * N + d] = fixed[m];
                continue;
            }
            int s = ghost_source(i, ny, i < 0 ? kind : c->bc[2], i < 0 ? c->bc[3] : kind, &fn, &ft);
            ptrdiff_t o = pidx(c, j, s);
            Qp[0 * N + d] = Qp[0 * N + o];
            Qp[1 * N + d] = ft ? -Qp[1 * N + o] : Qp[1 * N + o];
            Qp[2 * N + d] = fn ? -Qp[2 * N + o] : Qp[2 * N + o]; /* y momentum is normal */
            Qp[3 * N + d] = Qp[3 * N + o];
        }
    }
}

/* One face: the whole interface procedure of Secs. 2.1-2.4 at face j+1/2 of a
 * sweep. P[m] are the primitive planes in face-normal order (rho, un, ut, p);
 * `at` is the padded index of cell j, `s` the index step along the sweep and
 * `st` the step along the tangential direction; dn and dtn are the cell sizes
 * along and across the sweep. Writes the total flux (convective + viscous) in
 * face-normal order and the detector flag sigma. */
/* Primitive (rho, un, ut, p) dx-scaled gradient of a cell from its
 * conservative state q and conservative gradient dq (reading R20). */
static void prim_gradient_from_cons(double gamma, const double *q, const double *dq, double *dw)
{
    double rho = q[0], u = q[1] / rho, v = q[2] / rho;
    dw[0] = dq[0];
    dw[1] = (rho * dq[1] - q[1] * dq[0]) / (rho * rho); /* Sec. 2.2 chain rule */
    dw[2] = (rho * dq[2] - q[2] * dq[0]) / (rho * rho);
    dw[3] = (gamma - 1.0) * (dq[3] - u * dq[1] - v * dq[2] + 0.5 * (u * u + v * v) * dq[0]);
}

/* Left (rows of L) and right (columns of R) eigenvector matrices of the
 * x-direction flux Jacobian at the mean primitive state wb = (rho, u, v, p)
 * of a face, with c = sqrt(gamma p / rho).
 * cons = 0, reading R2 (end of Sec. 2.3, characteristic projection of the
 * primitive variables): the Jacobian of the primitive form U_t + A U_x = 0,
 * A = [[u, rho, 0, 0], [0, u, 0, 1/rho], [0, 0, u, 0], [0, rho c^2, 0, u]].
 * cons = 1, reading R20: the Jacobian dF/dQ of the conservative x-flux, with
 * H = c^2/(gamma-1) + (u^2+v^2)/2. Both diagonalise to (u-c, u, u, u+c). */
static void char_eigenvectors(int cons, double g, const double *wb, double Lm[4][4], double Rm[4][4])
{
    double rb = wb[0], pb = wb[3];
    double cb = sqrt(g * pb / rb);
    if (!cons) {
        const double L0[4][4] = {
            {0.0, -rb / (2.0 * cb), 0.0, 1.0 / (2.0 * cb * cb)},
            {1.0, 0.0, 0.0, -1.0 / (cb * cb)},
            {0.0, 0.0, 1.0, 0.0},
            {0.0, rb / (2.0 * cb), 0.0, 1.0 / (2.0 * cb * cb)},
        };
        const double R0[4][4] = {/* columns are the right eigenvectors */
                                 {1.0, 1.0, 0.0, 1.0},
                                 {-cb / rb, 0.0, 0.0, cb / rb},
                                 {0.0, 0.0, 1.0, 0.0},
                                 {cb * cb, 0.0, 0.0, cb * cb}};
        memcpy(Lm, L0, sizeof(L0));
        memcpy(Rm, R0, sizeof(R0));
    } else {
        double ub = wb[1], vb = wb[2];
        double q2 = ub * ub + vb * vb;
        double Hb = cb * cb / (g - 1.0) + 0.5 * q2;
        double b1 = (g - 1.0) / (cb * cb), b2 = 0.5 * q2 * b1;
        const double L1[4][4] = {
            {0.5 * (b2 + ub / cb), -0.5 * (b1 * ub + 1.0 / cb), -0.5 * b1 * vb, 0.5 * b1},
            {1.0 - b2, b1 * ub, b1 * vb, -b1},
            {-vb, 0.0, 1.0, 0.0},
            {0.5 * (b2 - ub / cb), -0.5 * (b1 * ub - 1.0 / cb), -0.5 * b1 * vb, 0.5 * b1},
        };
        const double R1[4][4] = {/* columns r1..r4 */
                                 {1.0, 1.0, 0.0, 1.0},
                                 {ub - cb, ub, 0.0, ub + cb},
                                 {vb, vb, 1.0, vb},
                                 {Hb - ub * cb, 0.5 * q2, vb, Hb + ub * cb}};
        memcpy(Lm, L1, sizeof(L1));
        memcpy(Rm, R1, sizeof(R1));
    }
}

static void face_flux(const or_cfg *c, const double *const P[4], const double *const Cq[4], ptrdiff_t at,
                      ptrdiff_t s, ptrdiff_t st, double dn, double dtn, double *Fh, int *sigma_out)
{
    const double g = c->gamma;
    const int order = c->order;
    double U[12][4]; /* U[k+5] = primitive state of cell j+k, k = -5..6 */
    double V[12][4]; /* the reconstructed variables: U (prim) or Q (cons) */
    for (int k = -5; k <= 6; ++k)
        for (int m = 0; m < 4; ++m) {
            U[k + 5][m] = P[m][at + k * s];
            V[k + 5][m] = c->cons ? Cq[m][at + k * s] : U[k + 5][m];
        }

    /* Eq. six: dx-scaled gradients of cells j-2..j+3 (D[k+2]) of the
     * reconstructed variables; DU: the primitive ones (viscous terms). */
    double D[6][4], DU[6][4];
    for (int k = -2; k <= 3; ++k) {
        for (int m = 0; m < 4; ++m) {
            double st7[7];
            for (int l = 0; l < 7; ++l)
                st7[l] = V[k + 5 - 3 + l][m];
            D[k + 2][m] = or_grad6(st7);
        }
        if (c->cons)
            prim_gradient_from_cons(g, V[k + 5], D[k + 2], DU[k + 2]);
        else
            for (int m = 0; m < 4; ++m)
                DU[k + 2][m] = D[k + 2][m];
    }

    /* Eqs. detector and buffer: sigma = 0 if min(psi_{j-2..j+3}) < psi_c. */
    double psimin = INFINITY;
    for (int k = -2; k <= 3; ++k) {
        double r5[5];
        for (int l = 0; l < 5; ++l)
            r5[l] = U[k + 5 - 2 + l][0];
        psimin = fmin(psimin, or_psi(r5));
    }
    int sigma = (psimin < 0.5) ? 0 : 1;
    *sigma_out = sigma;

    /* Reading R2: eigenvectors of the primitive Jacobian at the mean state
     * (R20: of the conservative Jacobian for MEG7-cons). */
    double wb[4] = {0.5 * (U[5][0] + U[6][0]), 0.5 * (U[5][1] + U[6][1]), 0.5 * (U[5][2] + U[6][2]),
                    0.5 * (U[5][3] + U[6][3])};
    double Lm[4][4], Rm[4][4];
    char_eigenvectors(c->cons, g, wb, Lm, Rm);
    /* characteristic values and gradients of cells j-2..j+3 */
    double Wc[6][4], Wd[6][4];
    for (int k = 0; k < 6; ++k) {
        for (int a = 0; a < 4; ++a) {
            double sv = 0.0, sd = 0.0;
            for (int b = 0; b < 4; ++b) {
                sv += Lm[a][b] * V[k + 3][b];
                sd += Lm[a][b] * D[k][b];
            }
            Wc[k][a] = sv;
            Wd[k][a] = sd;
        }
    }
    /* Eqs. grb, mp5Condition, alpha, mp-procedure per characteristic field */
    double wL[4], wR[4];
    for (int a = 0; a < 4; ++a) {
        double ph[5], dp[5];
        for (int k = 0; k < 5; ++k) { /* cells j-2..j+2 */
            ph[k] = Wc[k][a];
            dp[k] = Wd[k][a];
        }
        wL[a] = meg_left(order, ph, dp);
        for (int k = 0; k < 5; ++k) { /* cells j-1..j+3 */
            ph[k] = Wc[k + 1][a];
            dp[k] = Wd[k + 1][a];
        }
        wR[a] = meg_right(order, ph, dp);
    }
    double UL[4], UR[4];
    for (int b = 0; b < 4; ++b) {
        double sl = 0.0, sr = 0.0;
        for (int a = 0; a < 4; ++a) {
            sl += Rm[b][a] * wL[a];
            sr += Rm[b][a] * wR[a];
        }
        UL[b] = sl;
        UR[b] = sr;
    }
    if (c->cons) { /* the reconstructed face states are conservative */
        double qL[4], qR[4];
        memcpy(qL, UL, sizeof(qL));
        memcpy(qR, UR, sizeof(qR));
        cons_to_prim(g, qL, UL);
        cons_to_prim(g, qR, UR);
    }
    /* Reading R22: a face state with rho <= 0 or p <= 0 (characteristic
     * reconstruction across a strong shock, e.g. at the foot of the double
     * Mach reflection) is replaced by the adjacent cell's state. */
    if (!(UL[0] > 0.0 && UL[3] > 0.0))
        for (int m = 0; m < 4; ++m)
            UL[m] = U[5][m];
    if (!(UR[0] > 0.0 && UR[3] > 0.0))
        for (int m = 0; m < 4; ++m)
            UR[m] = U[6][m];

    /* Hybrid face fluxes (Sec. 2.4): F(f) of Eqs. flux-full/flux-right where
     * sigma = 1, F(Q_L), F(Q_R) of the MEG7 states where sigma = 0. */
    double FL[4], FR[4];
    if (sigma) {
        double fc[10][4]; /* cell fluxes of cells j-4..j+5 */
        for (int k = -4; k <= 5; ++k)
            euler_flux(g, U[k + 5], fc[k + 4]);
        for (int m = 0; m < 4; ++m) {
            double f9[9];
            for (int l = 0; l < 9; ++l)
                f9[l] = fc[l][m]; /* j-4..j+4 */
            FL[m] = flux_recon_left(order, f9);
            for (int l = 0; l < 9; ++l)
                f9[l] = fc[l + 1][m]; /* j-3..j+5 */
            FR[m] = flux_recon_right(order, f9);
        }
    } else {
        euler_flux(g, UL, FL);
        euler_flux(g, UR, FR);
    }
    hllc_face(g, c->riemann, UL, UR, FL, FR, Fh);

    if (c->mu > 0.0) {
        /* Sec. 2.1 with reading R8. T = gamma p / rho and its dx-scaled
         * gradient by the chain rule from rho' and p'. */
        const double av = 4.0, mu = c->mu;
        double T0 = g * U[5][3] / U[5][0], T1 = g * U[6][3] / U[6][0];
        double dT0 = g * (DU[2][3] / U[5][0] - U[5][3] * DU[2][0] / (U[5][0] * U[5][0]));
        double dT1 = g * (DU[3][3] / U[6][0] - U[6][3] * DU[3][0] / (U[6][0] * U[6][0]));
        /* Eq. alphad with Phi' = dx dPhi/dx: normal derivatives at the face */
        double un_n = 0.5 * (DU[2][1] + DU[3][1]) / dn + av / (2.0 * dn) * (U[6][1] - 0.5 * DU[3][1] - U[5][1] - 0.5 * DU[2][1]);
        double ut_n = 0.5 * (DU[2][2] + DU[3][2]) / dn + av / (2.0 * dn) * (U[6][2] - 0.5 * DU[3][2] - U[5][2] - 0.5 * DU[2][2]);
        double T_n = 0.5 * (dT0 + dT1) / dn + av / (2.0 * dn) * (T1 - 0.5 * dT1 - T0 - 0.5 * dT0);
        /* tangential derivatives: mean of the cell-centre sixth-order values */
        double tg[2][2];
        for (int q = 0; q < 2; ++q) {
            if (!c->cons) {
                for (int m = 1; m <= 2; ++m) {
                    double st7[7];
                    for (int l = 0; l < 7; ++l)
                        st7[l] = P[m][at + q * s + (l - 3) * st];
                    tg[q][m - 1] = or_grad6(st7) / dtn;
                }
            } else { /* chain rule from the conservative tangential gradients */
                double qc[4], dq[4], dw[4];
                for (int m = 0; m < 4; ++m) {
                    double st7[7];
                    for (int l = 0; l < 7; ++l)
                        st7[l] = Cq[m][at + q * s + (l - 3) * st];
                    dq[m] = or_grad6(st7);
                    qc[m] = Cq[m][at + q * s];
                }
                prim_gradient_from_cons(g, qc, dq, dw);
                tg[q][0] = dw[1] / dtn;
                tg[q][1] = dw[2] / dtn;
            }
        }
        double un_t = 0.5 * (tg[0][0] + tg[1][0]);
        double ut_t = 0.5 * (tg[0][1] + tg[1][1]);
        double unf = 0.5 * (U[5][1] + U[6][1]);
        double utf = 0.5 * (U[5][2] + U[6][2]);
        /* Eq. visc in the face-normal frame */
        double tau_nn = 2.0 / 3.0 * mu * (2.0 * un_n - ut_t);
        double tau_nt = mu * (un_t + ut_n);
        double q_n = -mu / (c->Pr * (g - 1.0)) * T_n;
        Fh[1] += -tau_nn;
        Fh[2] += -tau_nt;
        Fh[3] += -(tau_nn * unf + tau_nt * utf) + q_n;
    }
}

static int cfg_ok(const or_cfg *c)
{
    if (!c || c->nx < OR_G || c->ny < OR_G || !(c->dx > 0.0) || !(c->dy > 0.0) || !(c->gamma > 1.0) || c->mu < 0.0
        || !(c->Pr > 0.0))
        return 0;
    if (c->order != 7 && c->order != 4)
        return 0;
    if (c->cons != 0 && c->cons != 1)
        return 0;
    if (c->riemann != 0 && c->riemann != 1)
        return 0;
    for (int k = 0; k < 4; ++k) {
        if (c->bc[k] < 0 || c->bc[k] > OR_BC_CUSTOM)
            return 0;
        if (c->bc[k] == OR_BC_CUSTOM) {
            const int kk[2] = {c->side[k].kind_lo, c->side[k].kind_hi};
            for (int h = 0; h < 2; ++h)
                if (kk[h] != OR_BC_TRANSMISSIVE && kk[h] != OR_BC_NOSLIP_WALL && kk[h] != OR_BC_SYMMETRY
                    && kk[h] != OR_BC_FIXED)
                    return 0;
        }
    }
    if ((c->bc[0] == OR_BC_PERIODIC) != (c->bc[1] == OR_BC_PERIODIC))
        return 0;
    if ((c->bc[2] == OR_BC_PERIODIC) != (c->bc[3] == OR_BC_PERIODIC))
        return 0;
    return 1;
}

/* Eqs. eqn-differencing_residual and deriv: Res of the interior state Q
 * (SoA [4][ny][nx], x fastest) into Res (same layout). Optional outputs:
 * sigx [ny][nx+1] and sigy [ny+1][nx] detector flags per face. If mask
 * ([ny][nx]) is given, only cells with mask != 0 are evaluated (the others of
 * Res are left untouched). */
int or_residual(const or_cfg *c, const double *Q, double *Res, unsigned char *sigx, unsigned char *sigy,
                const unsigned char *mask)
{
    if (!cfg_ok(c) || !Q || !Res)
        return OR_ERR_ARG;
    const int nx = c->nx, ny = c->ny, W = nx + 2 * OR_G;
    const ptrdiff_t N = (ptrdiff_t)W * (ny + 2 * OR_G);
    double *Qp = (double *)malloc(sizeof(double) * 4 * N);
    double *Up = (double *)malloc(sizeof(double) * 4 * N);
    double *FX = (double *)malloc(sizeof(double) * 4 * (size_t)(nx + 1) * ny);
    double *FY = (double *)malloc(sizeof(double) * 4 * (size_t)nx * (ny + 1));
    if (!Qp || !Up || !FX || !FY) {
        free(Qp); free(Up); free(FX); free(FY);
        return OR_ERR_NOMEM;
    }
    for (int m = 0; m < 4; ++m)
        for (int i = 0; i < ny; ++i)
            for (int j = 0; j < nx; ++j)
                Qp[m * N + pidx(c, j, i)] = Q[((size_t)m * ny + i) * nx + j];
    or_fill_ghosts(c, Qp);
    /* Eq. pressure at every padded cell */
#pragma omp parallel for schedule(static)
    for (ptrdiff_t n = 0; n < N; ++n) {
        double q[4] = {Qp[n], Qp[N + n], Qp[2 * N + n], Qp[3 * N + n]}, w[4];
        cons_to_prim(c->gamma, q, w);
        for (int m = 0; m < 4; ++m)
            Up[m * N + n] = w[m];
    }
    const double *Px[4] = {Up, Up + N, Up + 2 * N, Up + 3 * N};     /* (rho, u, v, p) */
    const double *Py[4] = {Up, Up + 2 * N, Up + N, Up + 3 * N};     /* (rho, v, u, p) */
    const double *Cx[4] = {Qp, Qp + N, Qp + 2 * N, Qp + 3 * N};     /* (rho, rho u, rho v, E) */
    const double *Cy[4] = {Qp, Qp + 2 * N, Qp + N, Qp + 3 * N};     /* (rho, rho v, rho u, E) */

    /* x faces j+1/2, j = -1..nx-1, of every interior row */
#pragma omp parallel for schedule(dynamic, 1)
    for (int i = 0; i < ny; ++i) {
        for (int j = -1; j < nx; ++j) {
            if (mask) {
                int need = (j >= 0 && mask[(size_t)i * nx + j]) || (j + 1 < nx && mask[(size_t)i * nx + j + 1]);
                if (!need)
                    continue;
            }
            double fh[4];
            int sg;
            face_flux(c, Px, Cx, pidx(c, j, i), 1, W, c->dx, c->dy, fh, &sg);
            for (int m = 0; m < 4; ++m)
                FX[((size_t)m * ny + i) * (nx + 1) + (j + 1)] = fh[m];
            if (sigx)
                sigx[(size_t)i * (nx + 1) + (j + 1)] = (unsigned char)sg;
        }
    }
    /* y faces i+1/2, i = -1..ny-1, of every interior column */
#pragma omp parallel for schedule(dynamic, 1)
    for (int i = -1; i < ny; ++i) {
        for (int j = 0; j < nx; ++j) {
            if (mask) {
                int need = (i >= 0 && mask[(size_t)i * nx + j]) || (i + 1 < ny && mask[(size_t)(i + 1) * nx + j]);
                if (!need)
                    continue;
            }
            double fh[4];
            int sg;
            face_flux(c, Py, Cy, pidx(c, j, i), W, 1, c->dy, c->dx, fh, &sg);
            /* back from (rho, rho v, rho u, E) to (rho, rho u, rho v, E) */
            double gq[4] = {fh[0], fh[2], fh[1], fh[3]};
            for (int m = 0; m < 4; ++m)
                FY[((size_t)m * (ny + 1) + (i + 1)) * nx + j] = gq[m];
            if (sigy)
                sigy[(size_t)(i + 1) * nx + j] = (unsigned char)sg;
        }
    }
    /* Eq. deriv */
    for (int m = 0; m < 4; ++m) {
        for (int i = 0; i < ny; ++i) {
            for (int j = 0; j < nx; ++j) {
                if (mask && !mask[(size_t)i * nx + j])
                    continue;
                double dFdx = (FX[((size_t)m * ny + i) * (nx + 1) + j + 1] - FX[((size_t)m * ny + i) * (nx + 1) + j]) / c->dx;
                double dGdy = (FY[((size_t)m * (ny + 1) + i + 1) * nx + j] - FY[((size_t)m * (ny + 1) + i) * nx + j]) / c->dy;
                Res[((size_t)m * ny + i) * nx + j] = -dFdx - dGdy;
            }
        }
    }
    free(Qp);
    free(Up);
    free(FX);
    free(FY);
    return OR_OK;
}

/* Positivity check of one conservative state: rho > 0 and p > 0, finite. */
static int physical(double gamma, const double *q)
{
    double w[4];
    for (int m = 0; m < 4; ++m)
        if (!isfinite(q[m]))
            return 0;
    cons_to_prim(gamma, q, w);
    return w[0] > 0.0 && w[3] > 0.0;
}

/* Eq. rk: one third-order TVD Runge-Kutta step of size dt, in place on Q
 * (SoA [4][ny][nx]). Returns OR_ERR_NONPHYSICAL if any stage state has
 * rho <= 0, p <= 0 or a non-finite value (the step is still completed). */
int or_rk3_step(const or_cfg *c, double *Q, double dt)
{
    if (!cfg_ok(c) || !Q)
        return OR_ERR_ARG;
    const size_t n = (size_t)4 * c->nx * c->ny, cells = (size_t)c->nx * c->ny;
    double *Q0 = (double *)malloc(sizeof(double) * n);
    double *Qs = (double *)malloc(sizeof(double) * n);
    double *R = (double *)malloc(sizeof(double) * n);
    if (!Q0 || !Qs || !R) {
        free(Q0); free(Qs); free(R);
        return OR_ERR_NOMEM;
    }
    int rc = OR_OK, bad = 0;
    memcpy(Q0, Q, sizeof(double) * n);
    /* the stages see the boundaries at t, t + dt and t + dt/2 (Eq. rk) */
    or_cfg c2 = *c, c3 = *c;
    c2.t = c->t + dt;
    c3.t = c->t + 0.5 * dt;
    /* Q(1) = Qn + dt Res(Qn) */
    rc = or_residual(c, Q0, R, NULL, NULL, NULL);
    for (size_t k = 0; k < n && rc == OR_OK; ++k)
        Qs[k] = Q0[k] + dt * R[k];
    /* Q(2) = 3/4 Qn + 1/4 Q(1) + 1/4 dt Res(Q(1)) */
    for (size_t e = 0; e < cells && rc == OR_OK; ++e) {
        double q[4] = {Qs[e], Qs[cells + e], Qs[2 * cells + e], Qs[3 * cells + e]};
        bad |= !physical(c->gamma, q);
    }
    if (rc == OR_OK)
        rc = or_residual(&c2, Qs, R, NULL, NULL, NULL);
    for (size_t k = 0; k < n && rc == OR_OK; ++k)
        Qs[k] = 0.75 * Q0[k] + 0.25 * Qs[k] + 0.25 * dt * R[k];
    for (size_t e = 0; e < cells && rc == OR_OK; ++e) {
        double q[4] = {Qs[e], Qs[cells + e], Qs[2 * cells + e], Qs[3 * cells + e]};
        bad |= !physical(c->gamma, q);
    }
    /* Q(n+1) = 1/3 Qn + 2/3 Q(2) + 2/3 dt Res(Q(2)) */
    if (rc == OR_OK)
        rc = or_residual(&c3, Qs, R, NULL, NULL, NULL);
    for (size_t k = 0; k < n && rc == OR_OK; ++k)
        Q[k] = Q0[k] / 3.0 + 2.0 / 3.0 * Qs[k] + 2.0 / 3.0 * dt * R[k];
    for (size_t e = 0; e < cells && rc == OR_OK; ++e) {
        double q[4] = {Q[e], Q[cells + e], Q[2 * cells + e], Q[3 * cells + e]};
        bad |= !physical(c->gamma, q);
    }
    free(Q0);
    free(Qs);
    free(R);
    if (rc != OR_OK)
        return rc;
    return bad ? OR_ERR_NONPHYSICAL : OR_OK;
}

/* Sec. 2.5, the time-step formula written as dt = CFL / lambda with
 * lambda = max over cells of max((|u|+c)/dx, (|v|+c)/dy, alpha_v nu/dx^2,
 * alpha_v nu/dy^2), c = sqrt(gamma p / rho), nu = mu / rho, alpha_v = 4. */
double or_max_wavespeed(const or_cfg *c, const double *Q)
{
    const size_t cells = (size_t)c->nx * c->ny;
    double lam = 0.0;
    for (size_t e = 0; e < cells; ++e) {
        double q[4] = {Q[e], Q[cells + e], Q[2 * cells + e], Q[3 * cells + e]}, w[4];
        cons_to_prim(c->gamma, q, w);
        double cs = sqrt(c->gamma * w[3] / w[0]);
        double l = fmax((fabs(w[1]) + cs) / c->dx, (fabs(w[2]) + cs) / c->dy);
        if (c->mu > 0.0) {
            double nu = c->mu / w[0];
            l = fmax(l, fmax(4.0 * nu / (c->dx * c->dx), 4.0 * nu / (c->dy * c->dy)));
        }
        lam = fmax(lam, l);
    }
    return lam;
}

/* Training labels of the learned sensor: label[i][j] = 1 if the density
 * detector (Eq. detector with reading R4) marks interior cell (j, i) in x or
 * in y, i.e. psi_x < 0.5 or psi_y < 0.5 (the per-cell test before the buffer
 * of Eq. buffer). Q: interior state [4][ny][nx]. */
int or_trouble_labels(const or_cfg *c, const double *Q, unsigned char *label)
{
    if (!cfg_ok(c) || !Q || !label)
        return OR_ERR_ARG;
    const int nx = c->nx, ny = c->ny, W = nx + 2 * OR_G;
    const ptrdiff_t N = (ptrdiff_t)W * (ny + 2 * OR_G);
    double *Qp = (double *)malloc(sizeof(double) * 4 * N);
    if (!Qp)
        return OR_ERR_NOMEM;
    for (int m = 0; m < 4; ++m)
        for (int i = 0; i < ny; ++i)
            for (int j = 0; j < nx; ++j)
                Qp[m * N + pidx(c, j, i)] = Q[((size_t)m * ny + i) * nx + j];
    or_fill_ghosts(c, Qp);
    for (int i = 0; i < ny; ++i) {
        for (int j = 0; j < nx; ++j) {
            double rx[5], ry[5];
            for (int l = 0; l < 5; ++l) {
                rx[l] = Qp[pidx(c, j + l - 2, i)];
                ry[l] = Qp[pidx(c, j, i + l - 2)];
            }
            label[(size_t)i * nx + j] = (or_psi(rx) < 0.5 || or_psi(ry) < 0.5) ? 1 : 0;
        }
    }
    free(Qp);
    return OR_OK;
}

/* min(psi_x, psi_y) per interior cell ([ny][nx]): Eq. detector along x and
 * along y on the density, ghost cells by the boundary conditions. The cell is
 * a plain-detector cell (label 1) exactly when this is below psi_c = 0.5; the
 * learned sensor's soft training target is a function of it. */
int or_psi_min(const or_cfg *c, const double *Q, double *psi)
{
    if (!cfg_ok(c) || !Q || !psi)
        return OR_ERR_ARG;
    const int nx = c->nx, ny = c->ny, W = nx + 2 * OR_G;
    const ptrdiff_t N = (ptrdiff_t)W * (ny + 2 * OR_G);
    double *Qp = (double *)malloc(sizeof(double) * 4 * N);
    if (!Qp)
        return OR_ERR_NOMEM;
    for (int m = 0; m < 4; ++m)
        for (int i = 0; i < ny; ++i)
            for (int j = 0; j < nx; ++j)
                Qp[m * N + pidx(c, j, i)] = Q[((size_t)m * ny + i) * nx + j];
    or_fill_ghosts(c, Qp);
    for (int i = 0; i < ny; ++i) {
        for (int j = 0; j < nx; ++j) {
            double rx[5], ry[5];
            for (int l = 0; l < 5; ++l) {
                rx[l] = Qp[pidx(c, j + l - 2, i)];
                ry[l] = Qp[pidx(c, j, i + l - 2)];
            }
            const double px = or_psi(rx), py = or_psi(ry);
            psi[(size_t)i * nx + j] = px < py ? px : py;
        }
    }
    free(Qp);
    return OR_OK;
}

/* Pin helpers: the eigenvector matrices face_flux uses (char_eigenvectors),
 * L row-major (rows = left eigenvectors), R row-major (columns = right
 * eigenvectors), at primitive state w. */
void or_prim_eigenvectors(double g, const double *w, double *L, double *R)
{
    double Lm[4][4], Rm[4][4];
    char_eigenvectors(0, g, w, Lm, Rm);
    memcpy(L, Lm, sizeof(Lm));
    memcpy(R, Rm, sizeof(Rm));
}

void or_cons_eigenvectors(double g, const double *w, double *L, double *R)
{
    double Lm[4][4], Rm[4][4];
    char_eigenvectors(1, g, w, Lm, Rm);
    memcpy(L, Lm, sizeof(Lm));
    memcpy(R, Rm, sizeof(Rm));
}

/* Pin helper: fill ghosts of a padded state given as 4 planes of
 * (nx+2G) x (ny+2G) (exported so tests can check the boundary conditions). */
int or_fill_ghosts_padded(const or_cfg *c, double *Qp)
{
    if (!cfg_ok(c) || !Qp)
        return OR_ERR_ARG;
    or_fill_ghosts(c, Qp);
    return OR_OK;
}

int or_ghost_layers(void) { return OR_G; }

/* Number of OpenMP threads the oracle uses (1 without OpenMP). */
#ifdef _OPENMP
#include <omp.h>
int or_num_threads(void) { return omp_get_max_threads(); }
void or_set_num_threads(int n) { if (n > 0) omp_set_num_threads(n); }
#else
int or_num_threads(void) { return 1; }
void or_set_num_threads(int n) { (void)n; }
#endif
