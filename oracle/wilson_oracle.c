/*
 * wilson_oracle.c -- plain, slow, FP64 CPU oracle for the Wilson and
 * domain-wall Dirac operators and for conjugate gradient on their normal
 * equations.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library product links or calls
 * this file; only the tests, the smoke check and the benchmark's CPU-baseline
 * leg do.  It shares no code, header or constant with the CUDA path.
 *
 * What it computes.  The paper (Huth, Meyer, Wettig, Lattice 2019) benchmarks
 * "the Wilson Dirac operator" (Sec. 3.3, Fig. 4d) on top of Grid's stencil and
 * shift machinery (Sec. 3.1), but never writes the operator down.  This file
 * therefore writes out the textbook definitions, with every convention stated
 * once here:
 *
 *  - Lattice: dims L0..L3 (x, y, z, t), lexi(x) = x0 + L0*(x1 + L1*(x2 + L2*x3)).
 *    A hop that crosses the boundary in direction mu is multiplied by bc[mu]
 *    (+1 periodic, -1 antiperiodic).
 *  - Euclidean chiral gamma basis, 2x2 blocks, sigma_k the Pauli matrices:
 *      gamma_k = [[0, -i sigma_k], [i sigma_k, 0]]  (k = x, y, z),
 *      gamma_t = [[0, 1], [1, 0]],  gamma_5 = gamma_x gamma_y gamma_z gamma_t.
 *  - Wilson operator:
 *      (D psi)(x) = (m + 4r) psi(x) - 1/2 H psi(x),
 *      (H psi)(x) = sum_mu [ (r - gamma_mu) U_mu(x) psi(x+mu)
 *                          + (r + gamma_mu) U_mu(x-mu)^dag psi(x-mu) ],
 *    D^dag = gamma_5 D gamma_5, i.e. the same with r -/+ gamma swapped.
 *  - Even-odd: parity = (x0+x1+x2+x3) mod 2, a half field stores the sites of
 *    one parity at cb = lexi/2.  With a = m + 4r the even Schur complement is
 *      Mhat = a - (1/(4a)) H_eo H_oe,   Mhat^dag = a - (1/(4a)) H^dag_eo H^dag_oe.
 *  - Shamir domain wall (r = 1, same U on every slice, P+- = (1 +- gamma_5)/2):
 *      (D_dw psi)(s) = D_W(-M5) psi(s) + psi(s) - P- psi(s+1) - P+ psi(s-1),
 *    where P- psi(Ls) is read as -mf P- psi(0) and P+ psi(-1) as
 *    -mf P+ psi(Ls-1); D_dw^dag swaps P+ and P- and uses D_W^dag.
 *  - CG (Hestenes-Stiefel) on A x = b with A = K^dag K for K = D, Mhat, D_dw or
 *    the domain-wall Mhat,
 *    x0 = 0, stopping when |r|/|b| < tol.
 *  - Moebius domain wall (b5, c5; b5 = 1, c5 = 0 is the Shamir form above), with
 *    S psi(s) = P- psi(s+1) + P+ psi(s-1) under the same walls (-mf):
 *      D_M psi = (b5 D_W(-M5) + 1) psi + (c5 D_W(-M5) - 1) S psi,
 *      D_M^dag psi = (b5 D_W^dag + 1) psi + S^dag (c5 D_W^dag - 1) psi.
 *  - Even-odd (4-d parity) Schur complement of the domain-wall operator.  With
 *    M5 the part of D_dw that stays on a 4-d site,
 *      (M5 psi)(s) = (5 - M5) psi(s) - P- psi(s+1) - P+ psi(s-1)   (walls as above),
 *    and M_eo = -1/2 H_eo, M_oe = -1/2 H_oe on every slice:
 *      Mhat = M5 - M_eo M5^{-1} M_oe   on even 5-d half fields,
 *      Mhat^dag = M5^dag - M_oe^dag (M5^dag)^{-1} M_eo^dag,
 *    the source eta_hat_e = eta_e - M_eo M5^{-1} eta_o and the odd half of the
 *    solution psi_o = M5^{-1} (eta_o - M_oe psi_e).  M5^{-1} is applied by
 *    Gaussian elimination of M5's dense (4 Ls) x (4 Ls) spin-slice matrix.
 *  - The same Schur decomposition of the Moebius operator.  With B = b5 + c5 S,
 *    D_M = D_W(-M5) B + 1 - S splits into the site-local part
 *      M5_M = (4 - M5) B + 1 - S
 *    and the parity-changing parts M_eo = -1/2 H_eo B, M_oe = -1/2 H_oe B
 *    (B acts first, before the hop); Mhat, the prepared source and the
 *    reconstruction take the formulas above with M5 -> M5_M.
 *  - The lattice-wide SU(3) product of the paper's matrix-matrix benchmark
 *    (Sec. 3.3, Fig. 4a-c): C(x) = A(x) B(x) for 3x3 complex matrices stored
 *    [x][row][col] as {re, im} pairs, each entry summed over k = 0, 1, 2 in
 *    that order.
 *
 * Spin matrices are applied as dense 4x4 products and colour as full 3x3
 * complex products: no spin projection, no link compression, no reuse.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

enum { ORC_OK = 0, ORC_ERR_ARG = -1, ORC_ERR_NOMEM = -2, ORC_NOT_CONVERGED = -3 };
enum { ORC_OP_WILSON = 0, ORC_OP_WILSON_EO = 1, ORC_OP_DWF = 2, ORC_OP_DWF_EO = 3 };

typedef struct {
    int dims[4];
    int bc[4];
    double mass;
    double r;
    int Ls;
    double M5;
    double mf;
} orc_params;

#define SPIN 4
#define COL 3
#define SITE_DOF (SPIN * COL) /* complex numbers per site */

/* ---------------------------------------------------------------- geometry */

static long orc_volume(const int d[4]) { return (long)d[0] * d[1] * d[2] * d[3]; }

static void site_coords(long site, const int d[4], int x[4])
{
    for (int mu = 0; mu < 4; ++mu) {
        x[mu] = (int)(site % d[mu]);
        site /= d[mu];
    }
}

static long site_index(const int x[4], const int d[4])
{
    return x[0] + (long)d[0] * (x[1] + (long)d[1] * (x[2] + (long)d[2] * x[3]));
}

static int site_parity(const int x[4]) { return (x[0] + x[1] + x[2] + x[3]) & 1; }

/* --------------------------------------------------------------- gammas */

static void pauli(int k, cplx s[2][2])
{
    memset(s, 0, sizeof(cplx) * 4);
    if (k == 0) { s[0][1] = 1; s[1][0] = 1; }
    if (k == 1) { s[0][1] = -I; s[1][0] = I; }
    if (k == 2) { s[0][0] = 1; s[1][1] = -1; }
}

static void matmul4(const cplx a[4][4], const cplx b[4][4], cplx c[4][4])
{
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            cplx s = 0;
            for (int k = 0; k < 4; ++k) s += a[i][k] * b[k][j];
            c[i][j] = s;
        }
}

/* gamma_mu for mu = 0..3 (x, y, z, t); mu = 4 gives gamma_5. */
void orc_gamma(int mu, cplx g[4][4])
{
    memset(g, 0, sizeof(cplx) * 16);
    if (mu >= 0 && mu < 3) {
        cplx s[2][2];
        pauli(mu, s);
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j) {
                g[i][2 + j] = -I * s[i][j];
                g[2 + i][j] = I * s[i][j];
            }
    } else if (mu == 3) {
        g[0][2] = g[1][3] = g[2][0] = g[3][1] = 1;
    } else if (mu == 4) {
        cplx a[4][4], b[4][4], t1[4][4], t2[4][4];
        orc_gamma(0, a);
        orc_gamma(1, b);
        matmul4(a, b, t1);
        orc_gamma(2, a);
        matmul4(t1, a, t2);
        orc_gamma(3, b);
        matmul4(t2, b, g);
    }
}

/* ------------------------------------------------------------ site algebra */

/* out[a][i] += c * sum_b sum_j P[a][b] M[i][j] v[b][j]  (M = U, or U^dag if adj). */
static void add_spin_colour(cplx out[SPIN][COL], cplx c, const cplx P[4][4], const cplx *M, int adj,
                            const cplx *v)
{
    cplx mv[SPIN][COL];
    for (int b = 0; b < SPIN; ++b)
        for (int i = 0; i < COL; ++i) {
            cplx s = 0;
            for (int j = 0; j < COL; ++j) {
                cplx m = adj ? conj(M[j * COL + i]) : M[i * COL + j];
                s += m * v[b * COL + j];
            }
            mv[b][i] = s;
        }
    for (int a = 0; a < SPIN; ++a)
        for (int i = 0; i < COL; ++i) {
            cplx s = 0;
            for (int b = 0; b < SPIN; ++b) s += P[a][b] * mv[b][i];
            out[a][i] += c * s;
        }
}

/* ------------------------------------------------------------ Wilson hop */

/*
 * out = H in on the full lattice (dagger: H^dag = gamma_5 H gamma_5).
 * in, out: [V][4][3] complex; U: [V][4][3][3] complex.  out must not alias in.
 */
void orc_wilson_hop(cplx *out, const cplx *in, const cplx *U, const int d[4], const int bc[4], double r,
                    int dagger)
{
    long V = orc_volume(d);
    cplx fwd[4][4][4], bwd[4][4][4];
    double s = dagger ? -1.0 : 1.0;
    for (int mu = 0; mu < 4; ++mu) {
        cplx g[4][4];
        orc_gamma(mu, g);
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b) {
                cplx id = (a == b) ? r : 0;
                fwd[mu][a][b] = id - s * g[a][b];
                bwd[mu][a][b] = id + s * g[a][b];
            }
    }
#pragma omp parallel for schedule(static)
    for (long site = 0; site < V; ++site) {
        int x[4];
        site_coords(site, d, x);
        cplx acc[SPIN][COL];
        memset(acc, 0, sizeof(acc));
        for (int mu = 0; mu < 4; ++mu) {
            int y[4];
            /* forward neighbour x + mu */
            memcpy(y, x, sizeof(y));
            double eta = 1.0;
            y[mu] = x[mu] + 1;
            if (y[mu] == d[mu]) { y[mu] = 0; eta = bc[mu]; }
            long yp = site_index(y, d);
            add_spin_colour(acc, eta, (const cplx(*)[4])fwd[mu], U + (site * 4 + mu) * 9, 0,
                            in + yp * SITE_DOF);
            /* backward neighbour x - mu, link U_mu(x - mu)^dag */
            memcpy(y, x, sizeof(y));
            eta = 1.0;
            y[mu] = x[mu] - 1;
            if (y[mu] < 0) { y[mu] = d[mu] - 1; eta = bc[mu]; }
            long ym = site_index(y, d);
            add_spin_colour(acc, eta, (const cplx(*)[4])bwd[mu], U + (ym * 4 + mu) * 9, 1,
                            in + ym * SITE_DOF);
        }
        memcpy(out + site * SITE_DOF, acc, sizeof(acc));
    }
}

/* out = D in = (m + 4r) in - 1/2 H in (dagger: D^dag). */
void orc_wilson_dslash(cplx *out, const cplx *in, const cplx *U, const int d[4], const int bc[4],
                       double mass, double r, int dagger)
{
    long n = orc_volume(d) * SITE_DOF;
    orc_wilson_hop(out, in, U, d, bc, r, dagger);
    double a = mass + 4.0 * r;
    for (long i = 0; i < n; ++i) out[i] = a * in[i] - 0.5 * out[i];
}

/*
 * Even-odd hop: out (sites of parity out_parity) = H in (sites of the other
 * parity).  Half fields hold [Vh][4][3] at cb = lexi/2.  Computed literally:
 * the input is embedded in a full field that is zero on the other parity, the
 * full hop is applied, and the output parity is read back.
 */
int orc_wilson_hop_eo(cplx *out, const cplx *in, const cplx *U, const int d[4], const int bc[4],
                      double r, int dagger, int out_parity)
{
    long V = orc_volume(d);
    cplx *fin = calloc((size_t)V * SITE_DOF, sizeof(cplx));
    cplx *fout = malloc((size_t)V * SITE_DOF * sizeof(cplx));
    if (!fin || !fout) { free(fin); free(fout); return ORC_ERR_NOMEM; }
    for (long site = 0; site < V; ++site) {
        int x[4];
        site_coords(site, d, x);
        if (site_parity(x) != out_parity)
            memcpy(fin + site * SITE_DOF, in + (site / 2) * SITE_DOF, SITE_DOF * sizeof(cplx));
    }
    orc_wilson_hop(fout, fin, U, d, bc, r, dagger);
    for (long site = 0; site < V; ++site) {
        int x[4];
        site_coords(site, d, x);
        if (site_parity(x) == out_parity)
            memcpy(out + (site / 2) * SITE_DOF, fout + site * SITE_DOF, SITE_DOF * sizeof(cplx));
    }
    free(fin);
    free(fout);
    return ORC_OK;
}

/* Even Schur complement: out_e = a in_e - 1/(4a) H_eo H_oe in_e (dagger: with H^dag). */
int orc_wilson_schur(cplx *out, const cplx *in, const cplx *U, const int d[4], const int bc[4],
                     double mass, double r, int dagger)
{
    long nh = orc_volume(d) / 2 * SITE_DOF;
    cplx *t = malloc((size_t)nh * sizeof(cplx));
    if (!t) return ORC_ERR_NOMEM;
    int rc = orc_wilson_hop_eo(t, in, U, d, bc, r, dagger, 1);
    if (rc == ORC_OK) rc = orc_wilson_hop_eo(out, t, U, d, bc, r, dagger, 0);
    double a = mass + 4.0 * r;
    for (long i = 0; i < nh; ++i) out[i] = a * in[i] - out[i] / (4.0 * a);
    free(t);
    return rc;
}

/* ------------------------------------------------------------ domain wall */

/* out[s] += c * P v[s'] for a dense 4x4 spin matrix P, colour untouched. */
static void add_spin(cplx *out, cplx c, const cplx P[4][4], const cplx *v, long nsites)
{
    for (long site = 0; site < nsites; ++site)
        for (int a = 0; a < 4; ++a)
            for (int i = 0; i < 3; ++i) {
                cplx s = 0;
                for (int b = 0; b < 4; ++b) s += P[a][b] * v[site * SITE_DOF + b * 3 + i];
                out[site * SITE_DOF + a * 3 + i] += c * s;
            }
}

/* 5-d fields [Ls][V][4][3].  out = D_dw in (dagger: D_dw^dag). */
int orc_dwf_dslash(cplx *out, const cplx *in, const cplx *U, const int d[4], const int bc[4], int Ls,
                   double M5, double mf, int dagger)
{
    long V = orc_volume(d);
    long n4 = V * SITE_DOF;
    cplx g5[4][4], Pp[4][4], Pm[4][4];
    orc_gamma(4, g5);
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) {
            cplx id = (a == b) ? 1.0 : 0.0;
            Pp[a][b] = 0.5 * (id + g5[a][b]);
            Pm[a][b] = 0.5 * (id - g5[a][b]);
        }
    /* non-dagger: P- couples to s+1, P+ to s-1; the dagger swaps them */
    const cplx(*Pup)[4] = dagger ? (const cplx(*)[4])Pp : (const cplx(*)[4])Pm;
    const cplx(*Pdn)[4] = dagger ? (const cplx(*)[4])Pm : (const cplx(*)[4])Pp;
    for (int s = 0; s < Ls; ++s) {
        cplx *o = out + s * n4;
        const cplx *v = in + s * n4;
        orc_wilson_dslash(o, v, U, d, bc, -M5, 1.0, dagger);
        for (long i = 0; i < n4; ++i) o[i] += v[i];
        int sp = s + 1, sm = s - 1;
        double cp = -1.0, cm = -1.0;
        if (sp == Ls) { sp = 0; cp = mf; }      /* -(-mf) */
        if (sm < 0) { sm = Ls - 1; cm = mf; }
        add_spin(o, cp, Pup, in + sp * n4, V);
        add_spin(o, cm, Pdn, in + sm * n4, V);
    }
    return ORC_OK;
}

/* ----------------------------------------------------- Moebius domain wall */

/* out = S in (dagger: S^dag) on 5-d fields [Ls][nsites][4][3]:
   S psi(s) = P- psi(s+1) + P+ psi(s-1), walls: P- psi(Ls) -> -mf P- psi(0), P+ psi(-1) -> -mf P+ psi(Ls-1). */
static void dwf_shift(cplx *out, const cplx *in, long nsites, int Ls, double mf, int dagger)
{
    cplx g5[4][4], Pp[4][4], Pm[4][4];
    orc_gamma(4, g5);
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) {
            cplx id = (a == b) ? 1.0 : 0.0;
            Pp[a][b] = 0.5 * (id + g5[a][b]);
            Pm[a][b] = 0.5 * (id - g5[a][b]);
        }
    const cplx(*Pup)[4] = dagger ? (const cplx(*)[4])Pp : (const cplx(*)[4])Pm;
    const cplx(*Pdn)[4] = dagger ? (const cplx(*)[4])Pm : (const cplx(*)[4])Pp;
    long n4 = nsites * SITE_DOF;
    memset(out, 0, (size_t)Ls * n4 * sizeof(cplx));
    for (int s = 0; s < Ls; ++s) {
        int sp = s + 1, sm = s - 1;
        double cp = 1.0, cm = 1.0;
        if (sp == Ls) { sp = 0; cp = -mf; }
        if (sm < 0) { sm = Ls - 1; cm = -mf; }
        add_spin(out + s * n4, cp, Pup, in + sp * n4, nsites);
        add_spin(out + s * n4, cm, Pdn, in + sm * n4, nsites);
    }
}

/* out = D_M in (dagger: D_M^dag), 5-d fields [Ls][V][4][3]. */
int orc_dwf_mobius_dslash(cplx *out, const cplx *in, const cplx *U, const int d[4], const int bc[4], int Ls,
                          double M5, double mf, double b5, double c5, int dagger)
{
    long V = orc_volume(d), n4 = V * SITE_DOF, n5 = (long)Ls * n4;
    cplx *t = malloc((size_t)n5 * sizeof(cplx)), *u = malloc((size_t)n5 * sizeof(cplx));
    if (!t || !u) { free(t); free(u); return ORC_ERR_NOMEM; }
    if (!dagger) {
        dwf_shift(t, in, V, Ls, mf, 0);                                  /* t = S in              */
        for (long i = 0; i < n5; ++i) u[i] = b5 * in[i] + c5 * t[i];      /* u = b5 in + c5 S in   */
        for (int s = 0; s < Ls; ++s)                                      /* out = D_W u           */
            orc_wilson_dslash(out + s * n4, u + s * n4, U, d, bc, -M5, 1.0, 0);
        for (long i = 0; i < n5; ++i) out[i] += in[i] - t[i];            /* + in - S in           */
    } else {
        for (int s = 0; s < Ls; ++s)                                      /* t = D_W^dag in        */
            orc_wilson_dslash(t + s * n4, in + s * n4, U, d, bc, -M5, 1.0, 1);
        for (long i = 0; i < n5; ++i) u[i] = c5 * t[i] - in[i];           /* u = (c5 D_W^dag - 1) in */
        dwf_shift(out, u, V, Ls, mf, 1);                                  /* out = S^dag u         */
        for (long i = 0; i < n5; ++i) out[i] += b5 * t[i] + in[i];       /* + (b5 D_W^dag + 1) in */
    }
    free(t);
    free(u);
    return ORC_OK;
}

/* ------------------------------------------- domain wall, even-odd (4-d) */

/* P+ and P- (dagger: swapped) as dense 4x4 matrices: Pup acts with psi(s+1), Pdn with psi(s-1). */
static void dwf_projectors(int dagger, cplx Pup[4][4], cplx Pdn[4][4])
{
    cplx g5[4][4];
    orc_gamma(4, g5);
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) {
            cplx id = (a == b) ? 1.0 : 0.0;
            cplx pp = 0.5 * (id + g5[a][b]), pm = 0.5 * (id - g5[a][b]);
            Pup[a][b] = dagger ? pp : pm;
            Pdn[a][b] = dagger ? pm : pp;
        }
}

/* out = M5 in (dagger: M5^dag) on 5-d fields [Ls][nsites][4][3] of any site subset. */
void orc_dwf_m5(cplx *out, const cplx *in, long nsites, int Ls, double M5, double mf, int dagger)
{
    cplx Pup[4][4], Pdn[4][4];
    dwf_projectors(dagger, Pup, Pdn);
    long n4 = nsites * SITE_DOF;
    for (int s = 0; s < Ls; ++s) {
        cplx *o = out + s * n4;
        const cplx *v = in + s * n4;
        for (long i = 0; i < n4; ++i) o[i] = (5.0 - M5) * v[i];
        int sp = s + 1, sm = s - 1;
        double cp = -1.0, cm = -1.0;
        if (sp == Ls) { sp = 0; cp = mf; }
        if (sm < 0) { sm = Ls - 1; cm = mf; }
        add_spin(o, cp, Pup, in + sp * n4, nsites);
        add_spin(o, cm, Pdn, in + sm * n4, nsites);
    }
}

/* A site-local 5-d operator: out = A in on [Ls][nsites][4][3], parameters prm. */
typedef void (*site_op_fn)(cplx *out, const cplx *in, long nsites, int Ls, const double *prm, int dagger);

/* out = A^{-1} in for a site-local operator A that is the same (4 Ls) x (4 Ls)
   matrix on the (slice, spin) index of every site and colour: the matrix is
   built from A applied to unit vectors, factorised once by Gaussian
   elimination with partial pivoting, and solved for every (site, colour). */
static int site_op_inv(cplx *out, const cplx *in, long nsites, int Ls, site_op_fn op, const double *prm,
                       int dagger)
{
    if (Ls < 1 || Ls > 64) return ORC_ERR_ARG;
    const int n = 4 * Ls;
    cplx *A = calloc((size_t)n * n, sizeof(cplx));
    cplx *e = calloc((size_t)Ls * SITE_DOF, sizeof(cplx));
    cplx *col = malloc((size_t)Ls * SITE_DOF * sizeof(cplx));
    int *piv = malloc((size_t)n * sizeof(int));
    if (!A || !e || !col || !piv) { free(A); free(e); free(col); free(piv); return ORC_ERR_NOMEM; }
    /* column j = (s', b) of A: the operator applied to the unit vector at slice s', spin b, colour 0 (one site) */
    for (int j = 0; j < n; ++j) {
        memset(e, 0, (size_t)Ls * SITE_DOF * sizeof(cplx));
        e[(j / 4) * SITE_DOF + (j % 4) * 3] = 1.0;
        op(col, e, 1, Ls, prm, dagger);
        for (int i = 0; i < n; ++i) A[i * n + j] = col[(i / 4) * SITE_DOF + (i % 4) * 3];
    }
    /* LU with partial pivoting, in place */
    for (int k = 0; k < n; ++k) {
        int p = k;
        for (int i = k + 1; i < n; ++i)
            if (cabs(A[i * n + k]) > cabs(A[p * n + k])) p = i;
        piv[k] = p;
        if (p != k)
            for (int j = 0; j < n; ++j) { cplx t = A[k * n + j]; A[k * n + j] = A[p * n + j]; A[p * n + j] = t; }
        if (A[k * n + k] == 0) { free(A); free(e); free(col); free(piv); return ORC_ERR_ARG; }
        for (int i = k + 1; i < n; ++i) {
            cplx f = A[i * n + k] / A[k * n + k];
            A[i * n + k] = f;
            for (int j = k + 1; j < n; ++j) A[i * n + j] -= f * A[k * n + j];
        }
    }
    long n4 = nsites * SITE_DOF;
#pragma omp parallel for schedule(static)
    for (long site = 0; site < nsites; ++site) {
        for (int c = 0; c < 3; ++c) {
            cplx y[4 * 64];
            for (int i = 0; i < n; ++i) y[i] = in[(i / 4) * n4 + site * SITE_DOF + (i % 4) * 3 + c];
            for (int k = 0; k < n; ++k)
                if (piv[k] != k) { cplx t = y[k]; y[k] = y[piv[k]]; y[piv[k]] = t; }
            for (int i = 1; i < n; ++i)
                for (int j = 0; j < i; ++j) y[i] -= A[i * n + j] * y[j];
            for (int i = n - 1; i >= 0; --i) {
                for (int j = i + 1; j < n; ++j) y[i] -= A[i * n + j] * y[j];
                y[i] /= A[i * n + i];
            }
            for (int i = 0; i < n; ++i) out[(i / 4) * n4 + site * SITE_DOF + (i % 4) * 3 + c] = y[i];
        }
    }
    free(A);
    free(e);
    free(col);
    free(piv);
    return ORC_OK;
}

static void shamir_m5_op(cplx *out, const cplx *in, long nsites, int Ls, const double *prm, int dagger)
{
    orc_dwf_m5(out, in, nsites, Ls, prm[0], prm[1], dagger);
}

/* out = M5^{-1} in (dagger: (M5^dag)^{-1}). */
int orc_dwf_m5_inv(cplx *out, const cplx *in, long nsites, int Ls, double M5, double mf, int dagger)
{
    const double prm[2] = {M5, mf};
    return site_op_inv(out, in, nsites, Ls, shamir_m5_op, prm, dagger);
}

/* -1/2 H between parities on every slice of a 5-d half field [Ls][V/2][4][3]. */
static int dwf_hop_eo(cplx *out, const cplx *in, const cplx *U, const int d[4], const int bc[4], int Ls,
                      int dagger, int out_parity)
{
    long nh = orc_volume(d) / 2 * SITE_DOF;
    for (int s = 0; s < Ls; ++s) {
        int rc = orc_wilson_hop_eo(out + s * nh, in + s * nh, U, d, bc, 1.0, dagger, out_parity);
        if (rc != ORC_OK) return rc;
        for (long i = 0; i < nh; ++i) out[s * nh + i] *= -0.5;
    }
    return ORC_OK;
}

/* Mhat in_e (dagger: Mhat^dag) on even 5-d half fields. */
int orc_dwf_schur(cplx *out, const cplx *in, const cplx *U, const int d[4], const int bc[4], int Ls, double M5,
                  double mf, int dagger)
{
    long Vh = orc_volume(d) / 2, n5 = (long)Ls * Vh * SITE_DOF;
    if (Ls < 1 || Ls > 64) return ORC_ERR_ARG;
    cplx *t = malloc((size_t)n5 * sizeof(cplx)), *u = malloc((size_t)n5 * sizeof(cplx));
    if (!t || !u) { free(t); free(u); return ORC_ERR_NOMEM; }
    int rc = dwf_hop_eo(t, in, U, d, bc, Ls, dagger, 1);                        /* t_o = M_oe in_e   */
    if (rc == ORC_OK) rc = orc_dwf_m5_inv(u, t, Vh, Ls, M5, mf, dagger);         /* u_o = M5^-1 t_o   */
    if (rc == ORC_OK) rc = dwf_hop_eo(t, u, U, d, bc, Ls, dagger, 0);            /* t_e = M_eo u_o    */
    if (rc == ORC_OK) {
        orc_dwf_m5(out, in, Vh, Ls, M5, mf, dagger);                             /* out = M5 in_e     */
        for (long i = 0; i < n5; ++i) out[i] -= t[i];
    }
    free(t);
    free(u);
    return rc;
}

/* a full 5-d field [Ls][V][4][3] <-> the half field [Ls][V/2][4][3] of one parity */
static void split_parity(cplx *half, const cplx *full, const int d[4], int Ls, int parity, int to_full)
{
    long V = orc_volume(d);
    for (int s = 0; s < Ls; ++s)
        for (long site = 0; site < V; ++site) {
            int x[4];
            site_coords(site, d, x);
            if (site_parity(x) != parity) continue;
            cplx *h = half + ((long)s * (V / 2) + site / 2) * SITE_DOF;
            cplx *f = (cplx *)full + ((long)s * V + site) * SITE_DOF;
            if (to_full) memcpy(f, h, SITE_DOF * sizeof(cplx));
            else memcpy(h, f, SITE_DOF * sizeof(cplx));
        }
}

/* bhat_e = eta_e - M_eo M5^{-1} eta_o (eta a full 5-d field, bhat_e an even half field). */
int orc_dwf_eo_prepare(cplx *bhat, const cplx *eta, const cplx *U, const int d[4], const int bc[4], int Ls,
                       double M5, double mf)
{
    long n5 = (long)Ls * orc_volume(d) / 2 * SITE_DOF;
    cplx *eo = malloc((size_t)n5 * sizeof(cplx)), *u = malloc((size_t)n5 * sizeof(cplx));
    if (!eo || !u) { free(eo); free(u); return ORC_ERR_NOMEM; }
    split_parity(eo, eta, d, Ls, 1, 0);
    split_parity(bhat, eta, d, Ls, 0, 0);
    int rc = orc_dwf_m5_inv(u, eo, orc_volume(d) / 2, Ls, M5, mf, 0);
    if (rc == ORC_OK) rc = dwf_hop_eo(eo, u, U, d, bc, Ls, 0, 0);
    if (rc == ORC_OK)
        for (long i = 0; i < n5; ++i) bhat[i] -= eo[i];
    free(eo);
    free(u);
    return rc;
}

/* psi (full 5-d field) from its even half x_e: psi_o = M5^{-1} (eta_o - M_oe x_e). */
int orc_dwf_eo_reconstruct(cplx *psi, const cplx *xe, const cplx *eta, const cplx *U, const int d[4],
                           const int bc[4], int Ls, double M5, double mf)
{
    long n5 = (long)Ls * orc_volume(d) / 2 * SITE_DOF;
    cplx *t = malloc((size_t)n5 * sizeof(cplx)), *eo = malloc((size_t)n5 * sizeof(cplx));
    if (!t || !eo) { free(t); free(eo); return ORC_ERR_NOMEM; }
    split_parity(eo, eta, d, Ls, 1, 0);
    int rc = dwf_hop_eo(t, xe, U, d, bc, Ls, 0, 1);
    if (rc == ORC_OK) {
        for (long i = 0; i < n5; ++i) eo[i] -= t[i];
        rc = orc_dwf_m5_inv(t, eo, orc_volume(d) / 2, Ls, M5, mf, 0);
    }
    if (rc == ORC_OK) {
        split_parity((cplx *)xe, psi, d, Ls, 0, 1);
        split_parity(t, psi, d, Ls, 1, 1);
    }
    free(t);
    free(eo);
    return rc;
}

/* -------------------------------------- Moebius domain wall, even-odd (4-d) */

/* With D_W = (4 - M5) - H/2 (H the 4-d hop between parities) and B = b5 + c5 S,
   the Moebius operator D_M = D_W B + 1 - S splits by 4-d parity into
     the site-local part     M5_M = (4 - M5) B + 1 - S,
     the parity-changing part M_eo = -H_eo B / 2,  M_oe = -H_oe B / 2,
   and Mhat = M5_M - M_eo M5_M^{-1} M_oe on the even sites.  The adjoints take
   S -> S^dag and H -> H^dag (H_eo^dag = (H^dag)_oe), with B^dag = b5 + c5 S^dag
   moved to the left of the hop. */

/* out = B in (dagger: B^dag); out and in distinct */
static void mobius_b(cplx *out, const cplx *in, long nsites, int Ls, double mf, double b5, double c5, int dagger)
{
    long n5 = (long)Ls * nsites * SITE_DOF;
    dwf_shift(out, in, nsites, Ls, mf, dagger);
    for (long i = 0; i < n5; ++i) out[i] = b5 * in[i] + c5 * out[i];
}

/* out = M5_M in (dagger: M5_M^dag) on 5-d fields [Ls][nsites][4][3] of any site subset. */
void orc_dwf_mobius_m5(cplx *out, const cplx *in, long nsites, int Ls, double M5, double mf, double b5,
                       double c5, int dagger)
{
    long n5 = (long)Ls * nsites * SITE_DOF;
    dwf_shift(out, in, nsites, Ls, mf, dagger); /* out = S in */
    for (long i = 0; i < n5; ++i) out[i] = (4.0 - M5) * (b5 * in[i] + c5 * out[i]) + in[i] - out[i];
}

static void mobius_m5_op(cplx *out, const cplx *in, long nsites, int Ls, const double *prm, int dagger)
{
    orc_dwf_mobius_m5(out, in, nsites, Ls, prm[0], prm[1], prm[2], prm[3], dagger);
}

/* out = M5_M^{-1} in (dagger: (M5_M^dag)^{-1}). */
int orc_dwf_mobius_m5_inv(cplx *out, const cplx *in, long nsites, int Ls, double M5, double mf, double b5,
                          double c5, int dagger)
{
    const double prm[4] = {M5, mf, b5, c5};
    return site_op_inv(out, in, nsites, Ls, mobius_m5_op, prm, dagger);
}

/* Mhat in_e (dagger: Mhat^dag) on even 5-d half fields. */
int orc_dwf_mobius_schur(cplx *out, const cplx *in, const cplx *U, const int d[4], const int bc[4], int Ls,
                         double M5, double mf, double b5, double c5, int dagger)
{
    long Vh = orc_volume(d) / 2, n5 = (long)Ls * Vh * SITE_DOF;
    if (Ls < 1 || Ls > 64) return ORC_ERR_ARG;
    cplx *t = malloc((size_t)n5 * sizeof(cplx)), *u = malloc((size_t)n5 * sizeof(cplx));
    if (!t || !u) { free(t); free(u); return ORC_ERR_NOMEM; }
    int rc;
    if (!dagger) {
        mobius_b(u, in, Vh, Ls, mf, b5, c5, 0);                                    /* u_e = B in_e              */
        rc = dwf_hop_eo(t, u, U, d, bc, Ls, 0, 1);                                  /* t_o = M_oe in_e           */
        if (rc == ORC_OK) rc = orc_dwf_mobius_m5_inv(u, t, Vh, Ls, M5, mf, b5, c5, 0); /* u_o = M5^-1 t_o       */
        if (rc == ORC_OK) {
            mobius_b(t, u, Vh, Ls, mf, b5, c5, 0);                                  /* t_o = B u_o               */
            rc = dwf_hop_eo(u, t, U, d, bc, Ls, 0, 0);                              /* u_e = M_eo M5^-1 M_oe in_e */
        }
    } else {
        rc = dwf_hop_eo(u, in, U, d, bc, Ls, 1, 1);                                 /* u_o = -H_eo^dag in_e / 2  */
        if (rc == ORC_OK) {
            mobius_b(t, u, Vh, Ls, mf, b5, c5, 1);                                  /* t_o = M_eo^dag in_e       */
            rc = orc_dwf_mobius_m5_inv(u, t, Vh, Ls, M5, mf, b5, c5, 1);            /* u_o = M5^-dag t_o         */
        }
        if (rc == ORC_OK) rc = dwf_hop_eo(t, u, U, d, bc, Ls, 1, 0);                /* t_e = -H_oe^dag u_o / 2   */
        if (rc == ORC_OK) mobius_b(u, t, Vh, Ls, mf, b5, c5, 1);                    /* u_e = M_oe^dag u_o        */
    }
    if (rc == ORC_OK) {
        orc_dwf_mobius_m5(out, in, Vh, Ls, M5, mf, b5, c5, dagger);                 /* out = M5_M in_e           */
        for (long i = 0; i < n5; ++i) out[i] -= u[i];
    }
    free(t);
    free(u);
    return rc;
}

/* bhat_e = eta_e - M_eo M5_M^{-1} eta_o (eta a full 5-d field, bhat_e an even half field). */
int orc_dwf_mobius_eo_prepare(cplx *bhat, const cplx *eta, const cplx *U, const int d[4], const int bc[4], int Ls,
                              double M5, double mf, double b5, double c5)
{
    long Vh = orc_volume(d) / 2, n5 = (long)Ls * Vh * SITE_DOF;
    cplx *eo = malloc((size_t)n5 * sizeof(cplx)), *u = malloc((size_t)n5 * sizeof(cplx));
    if (!eo || !u) { free(eo); free(u); return ORC_ERR_NOMEM; }
    split_parity(eo, eta, d, Ls, 1, 0);
    split_parity(bhat, eta, d, Ls, 0, 0);
    int rc = orc_dwf_mobius_m5_inv(u, eo, Vh, Ls, M5, mf, b5, c5, 0); /* u_o = M5_M^-1 eta_o */
    if (rc == ORC_OK) {
        mobius_b(eo, u, Vh, Ls, mf, b5, c5, 0);                         /* B u_o               */
        rc = dwf_hop_eo(u, eo, U, d, bc, Ls, 0, 0);                     /* M_eo M5_M^-1 eta_o  */
    }
    if (rc == ORC_OK)
        for (long i = 0; i < n5; ++i) bhat[i] -= u[i];
    free(eo);
    free(u);
    return rc;
}

/* psi (full 5-d field) from its even half x_e: psi_o = M5_M^{-1} (eta_o - M_oe x_e). */
int orc_dwf_mobius_eo_reconstruct(cplx *psi, const cplx *xe, const cplx *eta, const cplx *U, const int d[4],
                                  const int bc[4], int Ls, double M5, double mf, double b5, double c5)
{
    long Vh = orc_volume(d) / 2, n5 = (long)Ls * Vh * SITE_DOF;
    cplx *t = malloc((size_t)n5 * sizeof(cplx)), *u = malloc((size_t)n5 * sizeof(cplx));
    cplx *eo = malloc((size_t)n5 * sizeof(cplx));
    if (!t || !u || !eo) { free(t); free(u); free(eo); return ORC_ERR_NOMEM; }
    split_parity(eo, eta, d, Ls, 1, 0);                                  /* eta_o                 */
    mobius_b(t, xe, Vh, Ls, mf, b5, c5, 0);                              /* t_e = B x_e           */
    int rc = dwf_hop_eo(u, t, U, d, bc, Ls, 0, 1);                       /* u_o = M_oe x_e        */
    if (rc == ORC_OK) {
        for (long i = 0; i < n5; ++i) eo[i] -= u[i];
        rc = orc_dwf_mobius_m5_inv(t, eo, Vh, Ls, M5, mf, b5, c5, 0);   /* t_o = M5_M^-1 (...)  */
    }
    if (rc == ORC_OK) {
        split_parity((cplx *)xe, psi, d, Ls, 0, 1);
        split_parity(t, psi, d, Ls, 1, 1);
    }
    free(t);
    free(u);
    free(eo);
    return rc;
}

/* ---------------------------------------------------------- normal ops, CG */

static long op_length(int op, const orc_params *p)
{
    long V = orc_volume(p->dims);
    if (op == ORC_OP_WILSON) return V * SITE_DOF;
    if (op == ORC_OP_WILSON_EO) return V / 2 * SITE_DOF;
    if (op == ORC_OP_DWF) return (long)p->Ls * V * SITE_DOF;
    if (op == ORC_OP_DWF_EO) return (long)p->Ls * (V / 2) * SITE_DOF;
    return -1;
}

/* out = K in (dagger: K^dag) for K = D, Mhat, D_dw or the domain-wall Mhat. */
int orc_apply_op(int op, cplx *out, const cplx *in, const cplx *U, const orc_params *p, int dagger)
{
    switch (op) {
    case ORC_OP_WILSON:
        orc_wilson_dslash(out, in, U, p->dims, p->bc, p->mass, p->r, dagger);
        return ORC_OK;
    case ORC_OP_WILSON_EO:
        return orc_wilson_schur(out, in, U, p->dims, p->bc, p->mass, p->r, dagger);
    case ORC_OP_DWF:
        return orc_dwf_dslash(out, in, U, p->dims, p->bc, p->Ls, p->M5, p->mf, dagger);
    case ORC_OP_DWF_EO:
        return orc_dwf_schur(out, in, U, p->dims, p->bc, p->Ls, p->M5, p->mf, dagger);
    }
    return ORC_ERR_ARG;
}

/* out = K^dag K in. */
int orc_apply_normal(int op, cplx *out, const cplx *in, const cplx *U, const orc_params *p)
{
    long n = op_length(op, p);
    if (n < 0) return ORC_ERR_ARG;
    cplx *t = malloc((size_t)n * sizeof(cplx));
    if (!t) return ORC_ERR_NOMEM;
    int rc = orc_apply_op(op, t, in, U, p, 0);
    if (rc == ORC_OK) rc = orc_apply_op(op, out, t, U, p, 1);
    free(t);
    return rc;
}

static double dot_re(const cplx *a, const cplx *b, long n)
{
    double s = 0;
    for (long i = 0; i < n; ++i) s += creal(conj(a[i]) * b[i]);
    return s;
}

/*
 * Conjugate gradient on K^dag K x = b from x = 0.  Returns ORC_OK when
 * |r|/|b| < tol within maxiter iterations (r the recursively updated
 * residual), ORC_NOT_CONVERGED otherwise; x holds the last iterate.
 */
int orc_cg(int op, cplx *x, const cplx *b, const cplx *U, const orc_params *p, double tol, int maxiter,
           int *iters, double *rel_res)
{
    long n = op_length(op, p);
    if (n < 0) return ORC_ERR_ARG;
    cplx *r = malloc((size_t)n * sizeof(cplx));
    cplx *q = malloc((size_t)n * sizeof(cplx));
    cplx *ap = malloc((size_t)n * sizeof(cplx));
    if (!r || !q || !ap) { free(r); free(q); free(ap); return ORC_ERR_NOMEM; }
    for (long i = 0; i < n; ++i) { x[i] = 0; r[i] = b[i]; q[i] = b[i]; }
    double bb = dot_re(b, b, n);
    double rr = bb;
    int k = 0, rc = ORC_NOT_CONVERGED;
    if (bb == 0.0) rc = ORC_OK;
    while (rc != ORC_OK && k < maxiter) {
        int e = orc_apply_normal(op, ap, q, U, p);
        if (e != ORC_OK) { rc = e; break; }
        double alpha = rr / dot_re(q, ap, n);
        for (long i = 0; i < n; ++i) { x[i] += alpha * q[i]; r[i] -= alpha * ap[i]; }
        double rr_new = dot_re(r, r, n);
        ++k;
        if (sqrt(rr_new / bb) < tol) { rr = rr_new; rc = ORC_OK; break; }
        double beta = rr_new / rr;
        rr = rr_new;
        for (long i = 0; i < n; ++i) q[i] = r[i] + beta * q[i];
    }
    if (iters) *iters = k;
    if (rel_res) *rel_res = bb > 0 ? sqrt(rr / bb) : 0.0;
    free(r);
    free(q);
    free(ap);
    return rc;
}

/* ------------------------------------------------- SU(3) x SU(3) product */

/* C[x] = A[x] B[x] for x < n: C_ij = sum_k A_ik B_kj (Sec. 3.3, Fig. 4a-c). */
void orc_su3_mul(cplx *C, const cplx *A, const cplx *B, long n)
{
#pragma omp parallel for schedule(static)
    for (long x = 0; x < n; ++x) {
        const cplx *a = A + 9 * x, *b = B + 9 * x;
        cplx *c = C + 9 * x;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                cplx t = 0;
                for (int k = 0; k < 3; ++k) t += a[3 * i + k] * b[3 * k + j];
                c[3 * i + j] = t;
            }
    }
}
