/*
 * z4c_oracle.c -- plain, slow, FP64 CPU oracle for the Z4c hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file; only the tests, the package's smoke check and the CPU
 * baseline leg of the benchmark do.  It shares no code, header, table or
 * helper with the CUDA path.  Build: gcc -O2 -ffp-contract=off -fopenmp
 * (see oracle/oracle.py).  No fused multiply-adds, no reassociation: every
 * sum is evaluated in the order written below.
 *
 * What it computes (paper: Zhu et al., "Performance-Portable Numerical
 * Relativity with AthenaK"):
 *   - Sec. 2: the vacuum Z4c system with Bona-Masso lapse and Gamma-driver
 *     shift.  The paper defers the continuum equations to GR-Athena++
 *     (Daszuta et al. 2021, Eqs. 8-13 and 22); the forms used here are the
 *     standard Z4c equations written out in rhs_point() below.
 *   - Sec. 3: Mesh of MeshBlocks with active + ghost regions; ghost zones
 *     filled from neighbouring blocks' active cells at every RK stage;
 *     cell-centred finite differences (Sec. 3.2).
 *   - Sec. 4.3: Kreiss-Oliger dissipation, constraint damping kappa1/kappa2,
 *     6th-order differencing and RK4.
 *
 * Readings taken where the paper is silent (numbered as in the design notes):
 *   R1 equation forms: as in rhs_point(); Gamma-tilde damping term is
 *      -2 alpha kappa1 (Gam - Gam_d); the K-gradient term in the Gam
 *      equation is -(1/3) gt^ij d_j (2 Khat + Theta); the evolved Gam is used
 *      only inside its derivative in the Ricci tensor, Gam_d elsewhere.
 *   R2 RK4 is the classic four-stage method; every stage state (and the
 *      final state) has the algebraic constraints enforced, then ghosts
 *      filled before its right-hand side is evaluated.
 *   R3 KO dissipation per direction: sigma (-1)^(N+1) / (2^(2N) h) times the
 *      centred 2N-th undivided difference, N = order/2 + 1 (2 for 2nd order,
 *      3 for 4th, 4 for 6th), so that the stencil reaches exactly the ghost
 *      width order/2 + 1.
 *   R4 mixed second derivatives are the tensor product of the centred first
 *      derivative stencils.
 *   R5 lopsided advection stencils for beta^k >= 0 lean towards +k; for
 *      beta^k < 0 the mirror image.  Order p uses offsets -(p/2-1)..p/2+1:
 *      -2..4 (6th), -1..3 (4th) and 0..2 (2nd, the one-sided 3-point
 *      difference; reading R19).
 *   R6 chi_g = max(chi, chi_floor) wherever 1/chi appears; chi itself is
 *      never clipped.
 *   R7 Sommerfeld outer boundary: every ghost cell whose centre lies outside
 *      the domain evolves du/dt = -(x^k d_k u + u - u_inf)/r, v = 1,
 *      u_inf = 1 for chi, alpha and the diagonal of gt, 0 otherwise, with
 *      2nd-order one-sided differences along each axis in which the cell
 *      index lies in the ghost range (pointing into the block), centred
 *      2nd-order differences otherwise.  Ghost copies never overwrite such a
 *      cell.
 *   R8 shift == 0 freezes beta (d_t beta = 0); lapse == 0 is harmonic
 *      slicing (mu_L = 1), lapse == 1 is 1+log (mu_L = 2/alpha).
 *   R12 mesh refinement (Sec. 3.1) on one address space: a coarse value is the
 *      active value of the coarser block that owns the point, or else the
 *      restriction of the same-level block that owns it; restriction takes
 *      5 fine cells per axis starting at 2c-1 (coarse cell c in the lower
 *      half of the block) or 2c-2 (upper half), clamped into the active
 *      region; prolongation takes the 5 coarse cells parent-2..parent+2.
 *   R13 along a non-periodic axis the 5 coarse cells of a prolongation
 *      stencil are shifted (by at most 2) to lie inside the domain, as the
 *      restriction stencil is kept inside the active region.
 *   R19 2nd-order differencing with 2 ghosts (Sec. 3.1 footnote): the
 *      transfer stencils take NP = N_g + 1 = 3 points per axis (3rd-order
 *      Lagrange, Sec. 3.1.1) instead of 5; restriction starts at 2c (lower
 *      half) or 2c-1 (upper half), prolongation takes parent-1..parent+1,
 *      shifted by at most 1 into the domain.  In general the starts are
 *      2c-(NP-3)/2, 2c-(NP-1)/2 and parent-(NP-1)/2.  3 and 4 ghosts keep
 *      NP = 5 (R12).
 *   R17 refinement indicators (Sec. 3.2): per block, min chi and max |grad
 *      chi| over interior cells, the gradient by the block's centred
 *      first-derivative stencil.
 *   R20 Psi4 (Sec. 3.3, computed with a coordinate tetrad; the paper gives no
 *      formulas): Psi4 = (E_ij - i B_ij) mb^i mb^j with the electric and
 *      magnetic parts of the Weyl tensor from the 3+1 variables (vacuum,
 *      K = Khat + 2 Theta) and mb = (e_th - i e_ph)/sqrt(2) from Gram-Schmidt
 *      on the radial, phi and theta coordinate vectors.  For a linear TT
 *      wave travelling along +x, on the +x axis, this is
 *      d_t^2 (h_yy - i h_yz) (h_zz = -h_yy); for one travelling along -x it
 *      vanishes.  See psi4_point().
 *   R18 puncture tracker (Sec. 3.3): dx/dt = -beta(x), one forward-Euler step
 *      per call, beta by 4-point Lagrange interpolation per axis.
 *
 * Field order (fixed): chi, gt_xx gt_xy gt_xz gt_yy gt_yz gt_zz, Khat,
 * At_xx .. At_zz, Gam^x Gam^y Gam^z, Theta, alpha, beta^x beta^y beta^z.
 *
 * Storage: for each block (in order) and each field, an (n_z+2g) x (n_y+2g)
 * x (n_x+2g) array, i fastest.  Blocks are concatenated.
 *
 * Parity status: every function below is pinned by tests in tests/ that
 * check it against closed forms, exact polynomial results, analytic
 * solutions and symmetries (see tests/test_oracle_*.py).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NF 22
enum {
  F_CHI = 0, F_GXX, F_GXY, F_GXZ, F_GYY, F_GYZ, F_GZZ, F_KHAT,
  F_AXX, F_AXY, F_AXZ, F_AYY, F_AYZ, F_AZZ, F_GAMX, F_GAMY, F_GAMZ,
  F_THETA, F_ALPHA, F_BETAX, F_BETAY, F_BETAZ
};

/* symmetric 3x3 index -> component 0..5 (xx xy xz yy yz zz) */
static const int SYM[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};

typedef struct {
  int32_t nblocks;
  int32_t ghosts;
  int32_t order;     /* 2, 4 or 6 */
  int32_t periodic;  /* 1: periodic box; 0: Sommerfeld outer boundary */
  int32_t lapse;     /* 0 harmonic, 1 one-plus-log */
  int32_t shift;     /* 0 frozen, 1 Gamma-driver */
  double dom_lo[3];
  double dom_hi[3];
  double ko_sigma;
  double kappa1;
  double kappa2;
  double eta;
  double chi_floor;
  const int32_t *n;  /* [nblocks][3] interior cells per direction */
  const double *lo;  /* [nblocks][3] lower corner of each active region */
  const double *h;   /* [nblocks] grid spacing */
  const int32_t *level; /* [nblocks] refinement level (h = h0 / 2^level), or NULL: all 0 */
} orc_mesh;

/* ------------------------------------------------------------------ */
/* storage geometry                                                    */
/* ------------------------------------------------------------------ */

static long ext(const orc_mesh *m, int b, int d) { return m->n[3 * b + d] + 2 * m->ghosts; }

static long blk_cells(const orc_mesh *m, int b) { return ext(m, b, 0) * ext(m, b, 1) * ext(m, b, 2); }

static long blk_offset(const orc_mesh *m, int b) {
  long off = 0;
  for (int q = 0; q < b; ++q) off += NF * blk_cells(m, q);
  return off;
}

long orc_state_size(const orc_mesh *m) { return blk_offset(m, m->nblocks); }

static void cell_centre(const orc_mesh *m, int b, int i, int j, int k, double x[3]) {
  int idx[3] = {i, j, k};
  for (int d = 0; d < 3; ++d) x[d] = m->lo[3 * b + d] + (idx[d] - m->ghosts + 0.5) * m->h[b];
}

static int is_interior(const orc_mesh *m, int b, int i, int j, int k) {
  int g = m->ghosts;
  return i >= g && i < m->n[3 * b] + g && j >= g && j < m->n[3 * b + 1] + g && k >= g &&
         k < m->n[3 * b + 2] + g;
}

/* centre outside the physical domain (only meaningful for non-periodic meshes) */
static int is_outside(const orc_mesh *m, const double x[3]) {
  for (int d = 0; d < 3; ++d)
    if (x[d] < m->dom_lo[d] || x[d] > m->dom_hi[d]) return 1;
  return 0;
}

/* Sommerfeld cell: ghost cell with centre outside a non-periodic domain (R7) */
static int is_sommerfeld(const orc_mesh *m, int b, int i, int j, int k) {
  if (m->periodic) return 0;
  if (is_interior(m, b, i, j, k)) return 0;
  double x[3];
  cell_centre(m, b, i, j, k, x);
  return is_outside(m, x);
}

/* ------------------------------------------------------------------ */
/* finite-difference stencils (Sec. 3; coefficients are the standard   */
/* centred / one-sided Taylor stencils, R3-R5)                         */
/* ------------------------------------------------------------------ */

typedef struct {
  const double *c;
  int len;
  int off; /* offset of c[0] relative to the centre */
  double den;
} stencil;

static const double C_D1_2[3] = {-1, 0, 1};
static const double C_D2_2[3] = {1, -2, 1};
static const double C_LP_2[3] = {-3, 4, -1};
static const double C_KO_2[5] = {1, -4, 6, -4, 1};
static const double C_D1_4[5] = {1, -8, 0, 8, -1};
static const double C_D1_6[7] = {-1, 9, -45, 0, 45, -9, 1};
static const double C_D2_4[5] = {-1, 16, -30, 16, -1};
static const double C_D2_6[7] = {2, -27, 270, -490, 270, -27, 2};
static const double C_LP_4[5] = {-3, -10, 18, -6, 1};
static const double C_LP_6[7] = {2, -24, -35, 80, -30, 8, -1};
static const double C_KO_4[7] = {1, -6, 15, -20, 15, -6, 1};
static const double C_KO_6[9] = {1, -8, 28, -56, 70, -56, 28, -8, 1};

static stencil st_d1(int order) {
  if (order == 2) return (stencil){C_D1_2, 3, -1, 2.0};
  stencil s = order == 4 ? (stencil){C_D1_4, 5, -2, 12.0} : (stencil){C_D1_6, 7, -3, 60.0};
  return s;
}
static stencil st_d2(int order) {
  if (order == 2) return (stencil){C_D2_2, 3, -1, 1.0};
  stencil s = order == 4 ? (stencil){C_D2_4, 5, -2, 12.0} : (stencil){C_D2_6, 7, -3, 180.0};
  return s;
}
static stencil st_lop(int order) {
  if (order == 2) return (stencil){C_LP_2, 3, 0, 2.0};
  stencil s = order == 4 ? (stencil){C_LP_4, 5, -1, 12.0} : (stencil){C_LP_6, 7, -2, 60.0};
  return s;
}
/* KO: den = 2^(2N); sign (-1)^(N+1) applied in ko() */
static stencil st_ko(int order) {
  if (order == 2) return (stencil){C_KO_2, 5, -2, 16.0};
  stencil s = order == 4 ? (stencil){C_KO_4, 7, -3, 64.0} : (stencil){C_KO_6, 9, -4, 256.0};
  return s;
}

static double apply(const double *p, long s, stencil st) {
  double acc = 0.0;
  for (int m = 0; m < st.len; ++m) acc += st.c[m] * p[(m + st.off) * s];
  return acc;
}

static double d1(const double *p, long s, int order, double h) {
  stencil st = st_d1(order);
  return apply(p, s, st) / (st.den * h);
}

static double d2(const double *p, long s, int order, double h) {
  stencil st = st_d2(order);
  return apply(p, s, st) / (st.den * h * h);
}

static double dmix(const double *p, long sa, long sb, int order, double h) {
  stencil st = st_d1(order);
  double acc = 0.0;
  for (int a = 0; a < st.len; ++a)
    for (int b = 0; b < st.len; ++b)
      acc += st.c[a] * st.c[b] * p[(a + st.off) * sa + (b + st.off) * sb];
  return acc / (st.den * st.den * h * h);
}

/* lopsided first derivative; upwind side chosen by the sign of beta (R5) */
static double dlop(const double *p, long s, int order, double h, double beta) {
  stencil st = st_lop(order);
  double acc = 0.0;
  if (beta >= 0.0) {
    acc = apply(p, s, st);
  } else {
    for (int m = 0; m < st.len; ++m) acc -= st.c[m] * p[-(m + st.off) * s];
  }
  return acc / (st.den * h);
}

static double ko(const double *p, long s, int order, double h, double sigma) {
  stencil st = st_ko(order);
  int N = order / 2 + 1;
  double sign = (N + 1) % 2 == 0 ? 1.0 : -1.0;
  return sign * sigma / (st.den * h) * apply(p, s, st);
}

/* Test hook: one finite-difference operator on an (nz,ny,nx) array.
 * kind 0: d/dx_dir1, 1: d2/dx_dir1^2, 2: d2/dx_dir1 dx_dir2,
 * 3: lopsided d/dx_dir1 with upwind sign of `arg`, 4: KO along dir1 with
 * sigma = `arg`. */
double orc_fd(int kind, int order, const double *f, int nx, int ny, int nz, int i, int j, int k,
              int dir1, int dir2, double h, double arg) {
  long st[3] = {1, nx, (long)nx * ny};
  const double *p = f + ((long)k * ny + j) * nx + i;
  (void)nz;
  switch (kind) {
    case 0: return d1(p, st[dir1], order, h);
    case 1: return d2(p, st[dir1], order, h);
    case 2: return dmix(p, st[dir1], st[dir2], order, h);
    case 3: return dlop(p, st[dir1], order, h, arg);
    case 4: return ko(p, st[dir1], order, h, arg);
    default: return NAN;
  }
}

/* ------------------------------------------------------------------ */
/* small linear algebra                                                */
/* ------------------------------------------------------------------ */

static double det3(const double g[3][3]) {
  return g[0][0] * (g[1][1] * g[2][2] - g[1][2] * g[2][1]) -
         g[0][1] * (g[1][0] * g[2][2] - g[1][2] * g[2][0]) +
         g[0][2] * (g[1][0] * g[2][1] - g[1][1] * g[2][0]);
}

/* inverse via adjugate / determinant */
static void inv3(const double g[3][3], double gi[3][3]) {
  double det = det3(g);
  gi[0][0] = (g[1][1] * g[2][2] - g[1][2] * g[2][1]) / det;
  gi[0][1] = (g[0][2] * g[2][1] - g[0][1] * g[2][2]) / det;
  gi[0][2] = (g[0][1] * g[1][2] - g[0][2] * g[1][1]) / det;
  gi[1][0] = (g[1][2] * g[2][0] - g[1][0] * g[2][2]) / det;
  gi[1][1] = (g[0][0] * g[2][2] - g[0][2] * g[2][0]) / det;
  gi[1][2] = (g[0][2] * g[1][0] - g[0][0] * g[1][2]) / det;
  gi[2][0] = (g[1][0] * g[2][1] - g[1][1] * g[2][0]) / det;
  gi[2][1] = (g[0][1] * g[2][0] - g[0][0] * g[2][1]) / det;
  gi[2][2] = (g[0][0] * g[1][1] - g[0][1] * g[1][0]) / det;
}

/* ------------------------------------------------------------------ */
/* Z4c right-hand side at one interior cell (Sec. 2, R1, R6, R8)       */
/* ------------------------------------------------------------------ */

typedef struct {
  /* values */
  double chi, Khat, Theta, alpha;
  double g[3][3], A[3][3], Gam[3], beta[3];
  /* derivatives: d?[k] = d_k ?, dd?[k][l] = d_k d_l ? */
  double dchi[3], dKhat[3], dTheta[3], dalpha[3];
  double dg[3][3][3];    /* dg[k][i][j] = d_k gt_ij */
  double dA[3][3][3];    /* dA[k][i][j] = d_k At_ij (constraints only) */
  double dbeta[3][3];    /* dbeta[k][i] = d_k beta^i */
  double dGam[3][3];     /* dGam[k][i] = d_k Gam^i */
  double ddchi[3][3], ddalpha[3][3];
  double ddg[3][3][3][3];  /* ddg[k][l][i][j] */
  double ddbeta[3][3][3];  /* ddbeta[k][l][i] */
} point_data;

static void gather_point(const orc_mesh *m, const double *c, long S, const long st[3], double h,
                         point_data *P, int need_dA) {
  int o = m->order;
  P->chi = c[F_CHI * S];
  P->Khat = c[F_KHAT * S];
  P->Theta = c[F_THETA * S];
  P->alpha = c[F_ALPHA * S];
  for (int i = 0; i < 3; ++i) {
    P->Gam[i] = c[(F_GAMX + i) * S];
    P->beta[i] = c[(F_BETAX + i) * S];
    for (int j = 0; j < 3; ++j) {
      P->g[i][j] = c[(F_GXX + SYM[i][j]) * S];
      P->A[i][j] = c[(F_AXX + SYM[i][j]) * S];
    }
  }
  for (int k = 0; k < 3; ++k) {
    P->dchi[k] = d1(c + F_CHI * S, st[k], o, h);
    P->dKhat[k] = d1(c + F_KHAT * S, st[k], o, h);
    P->dTheta[k] = d1(c + F_THETA * S, st[k], o, h);
    P->dalpha[k] = d1(c + F_ALPHA * S, st[k], o, h);
    for (int i = 0; i < 3; ++i) {
      P->dbeta[k][i] = d1(c + (F_BETAX + i) * S, st[k], o, h);
      P->dGam[k][i] = d1(c + (F_GAMX + i) * S, st[k], o, h);
      for (int j = 0; j < 3; ++j) {
        P->dg[k][i][j] = d1(c + (F_GXX + SYM[i][j]) * S, st[k], o, h);
        P->dA[k][i][j] = need_dA ? d1(c + (F_AXX + SYM[i][j]) * S, st[k], o, h) : 0.0;
      }
    }
    for (int l = 0; l < 3; ++l) {
      if (k == l) {
        P->ddchi[k][l] = d2(c + F_CHI * S, st[k], o, h);
        P->ddalpha[k][l] = d2(c + F_ALPHA * S, st[k], o, h);
      } else {
        P->ddchi[k][l] = dmix(c + F_CHI * S, st[k], st[l], o, h);
        P->ddalpha[k][l] = dmix(c + F_ALPHA * S, st[k], st[l], o, h);
      }
      for (int i = 0; i < 3; ++i) {
        const double *pb = c + (F_BETAX + i) * S;
        P->ddbeta[k][l][i] = k == l ? d2(pb, st[k], o, h) : dmix(pb, st[k], st[l], o, h);
        for (int j = 0; j < 3; ++j) {
          const double *pg = c + (F_GXX + SYM[i][j]) * S;
          P->ddg[k][l][i][j] = k == l ? d2(pg, st[k], o, h) : dmix(pg, st[k], st[l], o, h);
        }
      }
    }
  }
}

/* Geometry shared by the right-hand side and the constraints. */
typedef struct {
  double gi[3][3];        /* gt^ij */
  double Gl[3][3][3];     /* Gt_ijk = 1/2 (d_j g_ik + d_k g_ij - d_i g_jk) */
  double Gu[3][3][3];     /* Gt^i_jk */
  double Gd[3];           /* Gt_d^i = gt^jk Gt^i_jk */
  double R[3][3];         /* R_ij = Rt_ij + Rchi_ij */
  double Rs;              /* R = chi gt^ij R_ij */
  double Au[3][3];        /* At^ij */
  double AA;              /* At_ij At^ij */
  double K;               /* Khat + 2 Theta */
  double chig;            /* max(chi, chi_floor) */
} geometry;

static void compute_geometry(const orc_mesh *m, const point_data *P, geometry *G) {
  inv3(P->g, G->gi);
  G->chig = P->chi > m->chi_floor ? P->chi : m->chi_floor;
  G->K = P->Khat + 2.0 * P->Theta;

  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      for (int k = 0; k < 3; ++k)
        G->Gl[i][j][k] = 0.5 * (P->dg[j][i][k] + P->dg[k][i][j] - P->dg[i][j][k]);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      for (int k = 0; k < 3; ++k) {
        double s = 0.0;
        for (int l = 0; l < 3; ++l) s += G->gi[i][l] * G->Gl[l][j][k];
        G->Gu[i][j][k] = s;
      }
  for (int i = 0; i < 3; ++i) {
    double s = 0.0;
    for (int j = 0; j < 3; ++j)
      for (int k = 0; k < 3; ++k) s += G->gi[j][k] * G->Gu[i][j][k];
    G->Gd[i] = s;
  }

  /* conformal Ricci tensor Rt_ij */
  double Rt[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0.0;
      for (int l = 0; l < 3; ++l)
        for (int mm = 0; mm < 3; ++mm) s += -0.5 * G->gi[l][mm] * P->ddg[l][mm][i][j];
      for (int k = 0; k < 3; ++k)
        s += 0.5 * (P->g[k][i] * P->dGam[j][k] + P->g[k][j] * P->dGam[i][k]);
      for (int k = 0; k < 3; ++k) s += G->Gd[k] * 0.5 * (G->Gl[i][j][k] + G->Gl[j][i][k]);
      for (int l = 0; l < 3; ++l)
        for (int mm = 0; mm < 3; ++mm)
          for (int k = 0; k < 3; ++k)
            s += G->gi[l][mm] * (G->Gu[k][l][i] * G->Gl[j][k][mm] + G->Gu[k][l][j] * G->Gl[i][k][mm] +
                                 G->Gu[k][i][mm] * G->Gl[k][l][j]);
      Rt[i][j] = s;
    }

  /* conformal-factor part Rchi_ij */
  double ichi = 1.0 / G->chig;
  double DDchi[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = P->ddchi[i][j];
      for (int k = 0; k < 3; ++k) s -= G->Gu[k][i][j] * P->dchi[k];
      DDchi[i][j] = s;
    }
  double trDDchi = 0.0, dchi2 = 0.0;
  for (int l = 0; l < 3; ++l)
    for (int mm = 0; mm < 3; ++mm) {
      trDDchi += G->gi[l][mm] * DDchi[l][mm];
      dchi2 += G->gi[l][mm] * P->dchi[l] * P->dchi[mm];
    }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double Rchi = 0.5 * ichi * DDchi[i][j] + 0.5 * ichi * P->g[i][j] * trDDchi -
                    0.25 * ichi * ichi * (P->dchi[i] * P->dchi[j] + 3.0 * P->g[i][j] * dchi2);
      G->R[i][j] = Rt[i][j] + Rchi;
    }
  double s = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) s += G->gi[i][j] * G->R[i][j];
  G->Rs = P->chi * s;

  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double a = 0.0;
      for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) a += G->gi[i][k] * G->gi[j][l] * P->A[k][l];
      G->Au[i][j] = a;
    }
  double aa = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) aa += P->A[i][j] * G->Au[i][j];
  G->AA = aa;
}

static void rhs_point(const orc_mesh *m, const double *c, long S, const long st[3], double h,
                      double out[NF]) {
  point_data P;
  geometry G;
  gather_point(m, c, S, st, h, &P, 0);
  compute_geometry(m, &P, &G);
  const double al = P.alpha, chi = P.chi, K = G.K;
  const double k1 = m->kappa1, k2 = m->kappa2;
  const double ichi = 1.0 / G.chig;

  double divb = P.dbeta[0][0] + P.dbeta[1][1] + P.dbeta[2][2];

  /* physical second covariant derivative of the lapse and its trace */
  double DDa[3][3];
  double trgi_dchi_dal = 0.0;
  for (int k = 0; k < 3; ++k)
    for (int l = 0; l < 3; ++l) trgi_dchi_dal += G.gi[k][l] * P.dchi[k] * P.dalpha[l];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = P.ddalpha[i][j];
      for (int k = 0; k < 3; ++k) s -= G.Gu[k][i][j] * P.dalpha[k];
      s += 0.5 * ichi * (P.dchi[i] * P.dalpha[j] + P.dchi[j] * P.dalpha[i] - P.g[i][j] * trgi_dchi_dal);
      DDa[i][j] = s;
    }
  double lapl_a = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = P.ddalpha[i][j];
      for (int k = 0; k < 3; ++k) s -= G.Gu[k][i][j] * P.dalpha[k];
      lapl_a += chi * G.gi[i][j] * s;
    }
  lapl_a -= 0.5 * trgi_dchi_dal;

  /* chi */
  out[F_CHI] = 2.0 / 3.0 * chi * (al * K - divb);

  /* conformal metric */
  for (int i = 0; i < 3; ++i)
    for (int j = i; j < 3; ++j) {
      double s = -2.0 * al * P.A[i][j];
      for (int k = 0; k < 3; ++k) s += P.g[i][k] * P.dbeta[j][k] + P.g[j][k] * P.dbeta[i][k];
      s -= 2.0 / 3.0 * P.g[i][j] * divb;
      out[F_GXX + SYM[i][j]] = s;
    }

  /* Khat */
  out[F_KHAT] = -lapl_a + al * (G.AA + K * K / 3.0) + k1 * (1.0 - k2) * al * P.Theta;

  /* trace-free At */
  double X[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) X[i][j] = -DDa[i][j] + al * G.R[i][j];
  double trX = 0.0;
  for (int k = 0; k < 3; ++k)
    for (int l = 0; l < 3; ++l) trX += G.gi[k][l] * X[k][l];
  for (int i = 0; i < 3; ++i)
    for (int j = i; j < 3; ++j) {
      double s = 0.0;
      for (int k = 0; k < 3; ++k) s += P.A[i][k] * P.dbeta[j][k] + P.A[j][k] * P.dbeta[i][k];
      s -= 2.0 / 3.0 * P.A[i][j] * divb;
      s += chi * (X[i][j] - P.g[i][j] * trX / 3.0);
      double AikAkj = 0.0;
      for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) AikAkj += P.A[i][k] * G.gi[k][l] * P.A[l][j];
      s += al * (K * P.A[i][j] - 2.0 * AikAkj);
      out[F_AXX + SYM[i][j]] = s;
    }

  /* Theta */
  out[F_THETA] = 0.5 * al * (G.Rs - G.AA + 2.0 / 3.0 * K * K) - al * k1 * (2.0 + k2) * P.Theta;

  /* conformal connection functions */
  for (int i = 0; i < 3; ++i) {
    double s = 0.0;
    for (int k = 0; k < 3; ++k) s -= G.Gd[k] * P.dbeta[k][i];
    s += 2.0 / 3.0 * G.Gd[i] * divb;
    for (int j = 0; j < 3; ++j)
      for (int k = 0; k < 3; ++k) s += G.gi[j][k] * P.ddbeta[j][k][i];
    for (int j = 0; j < 3; ++j)
      for (int k = 0; k < 3; ++k) s += G.gi[i][j] * P.ddbeta[j][k][k] / 3.0;
    for (int j = 0; j < 3; ++j) s -= 2.0 * G.Au[i][j] * P.dalpha[j];
    double t = 0.0;
    for (int j = 0; j < 3; ++j)
      for (int k = 0; k < 3; ++k) t += G.Gu[i][j][k] * G.Au[j][k];
    for (int j = 0; j < 3; ++j) t -= 1.5 * ichi * G.Au[i][j] * P.dchi[j];
    for (int j = 0; j < 3; ++j) t -= G.gi[i][j] * (2.0 * P.dKhat[j] + P.dTheta[j]) / 3.0;
    s += 2.0 * al * t;
    s -= 2.0 * al * k1 * (P.Gam[i] - G.Gd[i]);
    out[F_GAMX + i] = s;
  }

  /* lapse (Bona-Masso) */
  if (m->lapse == 1)
    out[F_ALPHA] = -2.0 * al * P.Khat;
  else
    out[F_ALPHA] = -al * al * P.Khat;

  /* shift (Gamma-driver, integrated form) */
  for (int i = 0; i < 3; ++i) out[F_BETAX + i] = m->shift ? P.Gam[i] - m->eta * P.beta[i] : 0.0;

  /* advection along the shift (lopsided) and Kreiss-Oliger dissipation */
  int o = m->order;
  for (int f = 0; f < NF; ++f) {
    if (!m->shift && f >= F_BETAX) continue;
    const double *p = c + f * S;
    double adv = 0.0, diss = 0.0;
    for (int k = 0; k < 3; ++k) {
      adv += P.beta[k] * dlop(p, st[k], o, h, P.beta[k]);
      diss += ko(p, st[k], o, h, m->ko_sigma);
    }
    out[f] += adv + diss;
  }
}

/* Sommerfeld cell right-hand side (R7) */
static const double U_INF[NF] = {1, 1, 0, 0, 1, 0, 1, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 0, 0, 0};

static void sommerfeld_point(const orc_mesh *m, int b, const double *c, long S, const long st[3],
                             const int idx[3], double h, const double x[3], double out[NF]) {
  int g = m->ghosts;
  double r = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
  for (int f = 0; f < NF; ++f) {
    const double *p = c + f * S;
    double xdu = 0.0;
    for (int d = 0; d < 3; ++d) {
      long s = st[d];
      double du;
      if (idx[d] < g)
        du = (-3.0 * p[0] + 4.0 * p[s] - p[2 * s]) / (2.0 * h);
      else if (idx[d] >= m->n[3 * b + d] + g)
        du = (3.0 * p[0] - 4.0 * p[-s] + p[-2 * s]) / (2.0 * h);
      else
        du = (p[s] - p[-s]) / (2.0 * h);
      xdu += x[d] * du;
    }
    out[f] = -(xdu + p[0] - U_INF[f]) / r;
  }
}

/* Right-hand side of every evolved cell (interior + Sommerfeld) of every
 * block; other ghost cells get 0.  `u` must have its ghosts filled. */
void orc_rhs(const orc_mesh *m, const double *u, double *out) {
  long total = orc_state_size(m);
  memset(out, 0, sizeof(double) * total);
  for (int b = 0; b < m->nblocks; ++b) {
    long e0 = ext(m, b, 0), e1 = ext(m, b, 1), e2 = ext(m, b, 2);
    long S = e0 * e1 * e2;
    long st[3] = {1, e0, e0 * e1};
    const double *base = u + blk_offset(m, b);
    double *obase = out + blk_offset(m, b);
    double h = m->h[b];
#pragma omp parallel for schedule(dynamic, 1)
    for (long k = 0; k < e2; ++k) {
      double r[NF];
      for (long j = 0; j < e1; ++j)
        for (long i = 0; i < e0; ++i) {
          long cidx = (k * e1 + j) * e0 + i;
          if (is_interior(m, b, (int)i, (int)j, (int)k)) {
            rhs_point(m, base + cidx, S, st, h, r);
          } else if (is_sommerfeld(m, b, (int)i, (int)j, (int)k)) {
            double x[3];
            int idx[3] = {(int)i, (int)j, (int)k};
            cell_centre(m, b, (int)i, (int)j, (int)k, x);
            sommerfeld_point(m, b, base + cidx, S, st, idx, h, x, r);
          } else {
            continue;
          }
          for (int f = 0; f < NF; ++f) obase[f * S + cidx] = r[f];
        }
    }
  }
}

/* Right-hand side at a list of cells, cells[q] = (block, i, j, k) in storage
 * indices; out[q*NF + f].  Cells that are neither interior nor Sommerfeld
 * get 0. */
void orc_rhs_cells(const orc_mesh *m, const double *u, const int32_t *cells, long ncells, double *out) {
#pragma omp parallel for schedule(dynamic, 16)
  for (long q = 0; q < ncells; ++q) {
    int b = cells[4 * q], i = cells[4 * q + 1], j = cells[4 * q + 2], k = cells[4 * q + 3];
    long e0 = ext(m, b, 0), e1 = ext(m, b, 1), e2 = ext(m, b, 2);
    long S = e0 * e1 * e2;
    long st[3] = {1, e0, e0 * e1};
    long cidx = ((long)k * e1 + j) * e0 + i;
    const double *c = u + blk_offset(m, b) + cidx;
    double r[NF];
    if (is_interior(m, b, i, j, k)) {
      rhs_point(m, c, S, st, m->h[b], r);
    } else if (is_sommerfeld(m, b, i, j, k)) {
      double x[3];
      int idx[3] = {i, j, k};
      cell_centre(m, b, i, j, k, x);
      sommerfeld_point(m, b, c, S, st, idx, m->h[b], x, r);
    } else {
      for (int f = 0; f < NF; ++f) r[f] = 0.0;
    }
    for (int f = 0; f < NF; ++f) out[q * NF + f] = r[f];
  }
}

/* ------------------------------------------------------------------ */
/* ghost fill: same-level copies and periodic wrap (Sec. 3)            */
/* ------------------------------------------------------------------ */

/* owning block and storage index of the cell whose centre is x, or -1.
 * Blocks never overlap, so the block containing x is unique (whatever its
 * level). */
static int find_owner(const orc_mesh *m, const double x[3], int idx[3]) {
  for (int b = 0; b < m->nblocks; ++b) {
    int inside = 1;
    int q[3];
    for (int d = 0; d < 3; ++d) {
      double t = (x[d] - m->lo[3 * b + d]) / m->h[b];
      int c = (int)floor(t);
      if (c < 0 || c >= m->n[3 * b + d]) {
        inside = 0;
        break;
      }
      q[d] = c + m->ghosts;
    }
    if (inside) {
      for (int d = 0; d < 3; ++d) idx[d] = q[d];
      return b;
    }
  }
  return -1;
}

static int level_of(const orc_mesh *m, int b) { return m->level ? m->level[b] : 0; }

static void wrap(const orc_mesh *m, double x[3]) {
  for (int d = 0; d < 3; ++d) {
    double L = m->dom_hi[d] - m->dom_lo[d];
    while (x[d] < m->dom_lo[d]) x[d] += L;
    while (x[d] >= m->dom_hi[d]) x[d] -= L;
  }
}

/* Lagrange basis polynomial l_i(x) over the points xs[0..n-1] (Sec. 3.1.1) */
static double lagrange(const double *xs, int n, int i, double x) {
  double w = 1.0;
  for (int q = 0; q < n; ++q)
    if (q != i) w *= (x - xs[q]) / (xs[i] - xs[q]);
  return w;
}

/* Points per axis of the transfer stencils: N_g + 1 = 3 with 2 ghosts
 * (Sec. 3.1.1; reading R19), 5 otherwise (R12). */
static int transfer_points(const orc_mesh *m) { return m->ghosts == 2 ? 3 : 5; }

/* Restriction (Sec. 3.1.1): value of field f at the centre xc of a coarse
 * cell (spacing 2h) covered by fine block F, by NP-point Lagrange
 * interpolation per axis (3D tensor product) over fine cells that always lie
 * inside F's active region: the stencil starts at 2c-(NP-3)/2 for coarse
 * cells in the lower half of F and at 2c-(NP-1)/2 in the upper half (NP = 5:
 * 2c-1, 2c-2; NP = 3: 2c, 2c-1), clamped to [0, n-NP]. */
static double restrict_at(const orc_mesh *m, const double *u, int F, int f, const double xc[3]) {
  const double h = m->h[F];
  const int NP = transfer_points(m);
  int s[3];
  double w[3][5];
  for (int d = 0; d < 3; ++d) {
    int n = m->n[3 * F + d], nc = n / 2;
    int c = (int)floor((xc[d] - m->lo[3 * F + d]) / (2.0 * h));
    int st = c < nc / 2 ? 2 * c - (NP - 3) / 2 : 2 * c - (NP - 1) / 2;
    if (st < 0) st = 0;
    if (st > n - NP) st = n - NP;
    double xs[5];
    for (int q = 0; q < NP; ++q) xs[q] = m->lo[3 * F + d] + (st + q + 0.5) * h;
    for (int q = 0; q < NP; ++q) w[d][q] = lagrange(xs, NP, q, xc[d]);
    s[d] = st + m->ghosts;
  }
  long e0 = ext(m, F, 0), e1 = ext(m, F, 1), e2 = ext(m, F, 2);
  const double *base = u + blk_offset(m, F) + (long)f * e0 * e1 * e2;
  double v = 0.0;
  for (int c = 0; c < NP; ++c)
    for (int b = 0; b < NP; ++b)
      for (int a = 0; a < NP; ++a)
        v += w[2][c] * w[1][b] * w[0][a] * base[((long)(s[2] + c) * e1 + (s[1] + b)) * e0 + (s[0] + a)];
  return v;
}

/* Coarse value (all fields) at the centre xq of a level-lc cell: the active
 * value of the level-lc block that owns it, or the restriction of the
 * level-(lc+1) block that owns it (Sec. 3.1: coarse buffers hold the
 * restriction of the block's own / same-level neighbours' data and the
 * coarser neighbours' active data).  Returns 0, or 1 if no such value
 * exists (outside a non-periodic domain, or levels two apart). */
static int coarse_value(const orc_mesh *m, const double *u, const double xq_in[3], int lc, double v[NF]) {
  double xq[3] = {xq_in[0], xq_in[1], xq_in[2]};
  if (m->periodic)
    wrap(m, xq);
  else if (is_outside(m, xq))
    return 1;
  int idx[3];
  int N = find_owner(m, xq, idx);
  if (N < 0) return 1;
  if (level_of(m, N) == lc) {
    long e0 = ext(m, N, 0), e1 = ext(m, N, 1), e2 = ext(m, N, 2);
    for (int f = 0; f < NF; ++f)
      v[f] = u[blk_offset(m, N) + (long)f * e0 * e1 * e2 + ((long)idx[2] * e1 + idx[1]) * e0 + idx[0]];
    return 0;
  }
  if (level_of(m, N) == lc + 1) {
    for (int f = 0; f < NF; ++f) v[f] = restrict_at(m, u, N, f, xq);
    return 0;
  }
  return 1;
}

/* Ghost fill (Sec. 3, Sec. 3.1): every ghost cell of every block whose centre
 * lies inside the domain (or anywhere, periodic) gets, from the block that
 * owns that point,
 *   - same level: a copy of the active value;
 *   - one level finer: the restriction of the finer block's active data;
 *   - one level coarser: the prolongation, NP-point Lagrange per axis over
 *     the coarse cells parent-R..parent+R (R = (NP-1)/2: 2, or 1 with 2
 *     ghosts), evaluated at the fine centre (offset +-1/4 coarse spacing);
 *     along a non-periodic axis the NP cells are shifted to lie inside the
 *     domain (readings R13, R19); taken from the block's coarse buffer: the
 *     coarse values (coarse_value) over its extent widened by
 *     W = ceil(g/2) + R coarse cells (ghost depth plus stencil reach) on
 *     every side.
 * Ghost cells outside a non-periodic domain are Sommerfeld cells, untouched.
 * Returns 0, or -1 if a stencil needs data that is missing or two levels
 * apart. */
int orc_fill_ghosts(const orc_mesh *m, double *u) {
  int err = 0, oom = 0;
  /* blocks in parallel: each writes only its own ghost cells and reads only
   * active cells */
#pragma omp parallel for schedule(dynamic) reduction(| : err, oom)
  for (int b = 0; b < m->nblocks; ++b) {
    long e0 = ext(m, b, 0), e1 = ext(m, b, 1), e2 = ext(m, b, 2);
    long S = e0 * e1 * e2;
    double *base = u + blk_offset(m, b);
    const int L = level_of(m, b);
    const double hc = 2.0 * m->h[b];
    const int NP = transfer_points(m), RP = (NP - 1) / 2;
    const int W = (m->ghosts + 1) / 2 + RP;
    double *cb = NULL;   /* coarse buffer [cell][field], cells (nc+2W)^3 */
    char *cbad = NULL;
    long cbn[3] = {0, 0, 0}, cb0[3] = {0, 0, 0};
    for (long k = 0; k < e2; ++k)
      for (long j = 0; j < e1; ++j)
        for (long i = 0; i < e0; ++i) {
          if (is_interior(m, b, (int)i, (int)j, (int)k)) continue;
          double x[3], xw[3];
          cell_centre(m, b, (int)i, (int)j, (int)k, x);
          for (int d = 0; d < 3; ++d) xw[d] = x[d];
          if (m->periodic)
            wrap(m, xw);
          else if (is_outside(m, xw))
            continue; /* Sommerfeld cell: evolved, never filled */
          int q[3];
          int ob = find_owner(m, xw, q);
          if (ob < 0) continue;
          long cidx = (k * e1 + j) * e0 + i;
          int lo_ = level_of(m, ob);
          if (lo_ == L) {
            long f0 = ext(m, ob, 0), f1 = ext(m, ob, 1), f2 = ext(m, ob, 2);
            long So = f0 * f1 * f2;
            const double *src = u + blk_offset(m, ob) + ((long)q[2] * f1 + q[1]) * f0 + q[0];
            for (int f = 0; f < NF; ++f) base[f * S + cidx] = src[f * So];
          } else if (lo_ == L + 1) {
            for (int f = 0; f < NF; ++f) base[f * S + cidx] = restrict_at(m, u, ob, f, xw);
          } else if (lo_ == L - 1) {
            if (!cb) { /* build this block's coarse buffer on first use */
              long tot = 1;
              for (int d = 0; d < 3; ++d) {
                cb0[d] = (long)llround((m->lo[3 * b + d] - m->dom_lo[d]) / hc) - W;
                cbn[d] = m->n[3 * b + d] / 2 + 2 * W;
                tot *= cbn[d];
              }
              cb = malloc(sizeof(double) * NF * tot);
              cbad = malloc(tot);
              if (!cb || !cbad) {
                oom = 1;
                goto next_block;
              }
              for (long c2 = 0; c2 < cbn[2]; ++c2)
                for (long c1 = 0; c1 < cbn[1]; ++c1)
                  for (long c0 = 0; c0 < cbn[0]; ++c0) {
                    long ci = (c2 * cbn[1] + c1) * cbn[0] + c0;
                    double xq[3] = {m->dom_lo[0] + (cb0[0] + c0 + 0.5) * hc,
                                    m->dom_lo[1] + (cb0[1] + c1 + 0.5) * hc,
                                    m->dom_lo[2] + (cb0[2] + c2 + 0.5) * hc};
                    cbad[ci] = (char)coarse_value(m, u, xq, L - 1, cb + NF * ci);
                  }
            }
            long p[3];
            double w[3][5];
            for (int d = 0; d < 3; ++d) {
              /* stencil start (global level-(L-1) index): parent - RP,
               * shifted into a non-periodic domain (readings R13, R19) */
              long st = (long)floor((x[d] - m->dom_lo[d]) / hc) - RP;
              if (!m->periodic) {
                long nd = (long)llround((m->dom_hi[d] - m->dom_lo[d]) / hc);
                if (st > nd - NP) st = nd - NP;
                if (st < 0) st = 0;
              }
              p[d] = st + RP - cb0[d]; /* stencil centre, buffer index */
              double xs[5];
              for (int a = 0; a < NP; ++a) xs[a] = m->dom_lo[d] + (st + a + 0.5) * hc;
              for (int a = 0; a < NP; ++a) w[d][a] = lagrange(xs, NP, a, x[d]);
            }
            double v[NF];
            for (int f = 0; f < NF; ++f) v[f] = 0.0;
            for (int c = 0; c < NP; ++c)
              for (int bb = 0; bb < NP; ++bb)
                for (int a = 0; a < NP; ++a) {
                  long c0 = p[0] + a - RP, c1 = p[1] + bb - RP, c2 = p[2] + c - RP;
                  if (c0 < 0 || c1 < 0 || c2 < 0 || c0 >= cbn[0] || c1 >= cbn[1] || c2 >= cbn[2]) {
                    err = 1;
                    continue;
                  }
                  long ci = (c2 * cbn[1] + c1) * cbn[0] + c0;
                  if (cbad[ci]) err = 1;
                  double wt = w[2][c] * w[1][bb] * w[0][a];
                  for (int f = 0; f < NF; ++f) v[f] += wt * cb[NF * ci + f];
                }
            for (int f = 0; f < NF; ++f) base[f * S + cidx] = v[f];
          } else {
            err = 1;
          }
        }
  next_block:
    free(cb);
    free(cbad);
  }
  if (oom) return -3;
  return err ? -1 : 0;
}

/* ------------------------------------------------------------------ */
/* algebraic constraint enforcement: det gt = 1, tr At = 0              */
/* ------------------------------------------------------------------ */

static void enforce_cell(double *c, long S) {
  double g[3][3], A[3][3], gi[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      g[i][j] = c[(F_GXX + SYM[i][j]) * S];
      A[i][j] = c[(F_AXX + SYM[i][j]) * S];
    }
  double det = det3(g);
  double scale = pow(det, -1.0 / 3.0);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) g[i][j] *= scale;
  inv3(g, gi);
  double tr = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) tr += gi[i][j] * A[i][j];
  for (int i = 0; i < 3; ++i)
    for (int j = i; j < 3; ++j) {
      c[(F_GXX + SYM[i][j]) * S] = g[i][j];
      c[(F_AXX + SYM[i][j]) * S] = A[i][j] - g[i][j] * tr / 3.0;
    }
}

static int is_evolved(const orc_mesh *m, int b, int i, int j, int k) {
  return is_interior(m, b, i, j, k) || is_sommerfeld(m, b, i, j, k);
}

void orc_enforce(const orc_mesh *m, double *u) {
  for (int b = 0; b < m->nblocks; ++b) {
    long e0 = ext(m, b, 0), e1 = ext(m, b, 1), e2 = ext(m, b, 2);
    long S = e0 * e1 * e2;
    double *base = u + blk_offset(m, b);
    for (long k = 0; k < e2; ++k)
      for (long j = 0; j < e1; ++j)
        for (long i = 0; i < e0; ++i)
          if (is_evolved(m, b, (int)i, (int)j, (int)k)) enforce_cell(base + (k * e1 + j) * e0 + i, S);
  }
}

/* ------------------------------------------------------------------ */
/* classic RK4 (R2)                                                    */
/* ------------------------------------------------------------------ */

/* y = x + a * k on evolved cells */
static void axpy_evolved(const orc_mesh *m, double *y, const double *x, double a, const double *k) {
  for (int b = 0; b < m->nblocks; ++b) {
    long e0 = ext(m, b, 0), e1 = ext(m, b, 1), e2 = ext(m, b, 2);
    long S = e0 * e1 * e2;
    long off = blk_offset(m, b);
    for (long kk = 0; kk < e2; ++kk)
      for (long j = 0; j < e1; ++j)
        for (long i = 0; i < e0; ++i) {
          if (!is_evolved(m, b, (int)i, (int)j, (int)kk)) continue;
          long c = off + (kk * e1 + j) * e0 + i;
          for (int f = 0; f < NF; ++f) y[c + f * S] = x[c + f * S] + a * k[c + f * S];
        }
  }
}

int orc_rk4_step(const orc_mesh *m, double *u, double dt, int nsteps) {
  long n = orc_state_size(m);
  double *us = malloc(sizeof(double) * n);
  double *k[4];
  for (int s = 0; s < 4; ++s) k[s] = malloc(sizeof(double) * n);
  if (!us || !k[0] || !k[1] || !k[2] || !k[3]) return -1;
  const double c[4] = {0.0, 0.5, 0.5, 1.0};
  for (int step = 0; step < nsteps; ++step) {
    memcpy(us, u, sizeof(double) * n);
    for (int s = 0; s < 4; ++s) {
      if (s > 0) {
        axpy_evolved(m, us, u, c[s] * dt, k[s - 1]);
        orc_enforce(m, us);
      }
      if (orc_fill_ghosts(m, us)) return -2;
      orc_rhs(m, us, k[s]);
    }
    /* u+ = u0 + dt/6 (k1 + 2 k2 + 2 k3 + k4) */
    for (long q = 0; q < n; ++q) {
      double sum = k[0][q] + 2.0 * k[1][q] + 2.0 * k[2][q] + k[3][q];
      us[q] = sum;
    }
    axpy_evolved(m, u, u, dt / 6.0, us);
    orc_enforce(m, u);
  }
  free(us);
  for (int s = 0; s < 4; ++s) free(k[s]);
  return 0;
}

/* ------------------------------------------------------------------ */
/* constraints H and M^i and their norms                               */
/* ------------------------------------------------------------------ */

/* norms[0] = ||H||_2, [1] = ||M||_2, [2] = max|H|, [3] = ||H||_2 over
 * r > r_mask, [4] = ||M||_2 over r > r_mask, [5] = max|M|.
 * ||X||_2 = sqrt(sum X^2 h^3 / sum h^3) over interior cells.
 * per_cell (nullable): 4 values per storage cell (H, Mx, My, Mz), field
 * major like the state (4 "fields"). */
/* ------------------------------------------------------------------ */
/* Weyl scalar Psi4 on the grid (Sec. 3.3: the outgoing Weyl scalar in  */
/* a coordinate tetrad; reading R20)                                   */
/* ------------------------------------------------------------------ */

/* Psi4 = (E_ij - i B_ij) mb^i mb^j at one interior cell, with
 *   gamma_ij = gt_ij / chi_g,  K_ij = (At_ij + gt_ij K / 3) / chi_g,
 *   K = Khat + 2 Theta,
 *   E_ij = R_ij + K K_ij - K_ik gamma^kl K_lj      (R_ij: compute_geometry),
 *   B_ij = symmetric part of gamma_im eps^mkl D_k K_lj,
 *          eps^mkl = [mkl] / sqrt(det gamma),
 *   D_k K_lj = d_k K_lj - G^m_kl K_mj - G^m_kj K_lm with the Christoffels of
 *   gamma, G^m_kl = Gt^m_kl - (delta^m_k d_l chi + delta^m_l d_k chi -
 *   gt_kl gt^mn d_n chi) / (2 chi_g), and d_k K_lj by the product rule from
 *   the derivatives of At, gt, Khat, Theta and chi;
 *   mb = (e_th - i e_ph) / sqrt(2) from Gram-Schmidt in gamma on the
 *   coordinate vectors x^i (radial), (-y, x, 0) (phi) and
 *   (x z, y z, -(x^2 + y^2)) (theta), in that order.
 * x: the cell centre; the tetrad is undefined on the z axis, where the
 * result is 0. */
static void psi4_point(const orc_mesh *m, const double *c, long S, const long st[3], double h,
                       const double x[3], double out[2]) {
  out[0] = out[1] = 0.0;
  if (x[0] * x[0] + x[1] * x[1] == 0.0) return;
  point_data P;
  geometry G;
  gather_point(m, c, S, st, h, &P, 1);
  compute_geometry(m, &P, &G);
  const double ichi = 1.0 / G.chig, K = G.K;
  double gam[3][3], gamu[3][3], Kij[3][3], dK[3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      gam[i][j] = P.g[i][j] * ichi;
      gamu[i][j] = G.gi[i][j] * G.chig;
      Kij[i][j] = (P.A[i][j] + P.g[i][j] * K / 3.0) * ichi;
    }
  for (int k = 0; k < 3; ++k) dK[k] = P.dKhat[k] + 2.0 * P.dTheta[k];
  double dKij[3][3][3], Gam[3][3][3];
  for (int k = 0; k < 3; ++k)
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j)
        dKij[k][i][j] = (P.dA[k][i][j] + (P.dg[k][i][j] * K + P.g[i][j] * dK[k]) / 3.0) * ichi -
                        Kij[i][j] * P.dchi[k] * ichi;
  for (int mm = 0; mm < 3; ++mm)
    for (int k = 0; k < 3; ++k)
      for (int l = 0; l < 3; ++l) {
        double gd = 0.0;
        for (int n = 0; n < 3; ++n) gd += G.gi[mm][n] * P.dchi[n];
        double dk = (mm == k ? P.dchi[l] : 0.0) + (mm == l ? P.dchi[k] : 0.0) - P.g[k][l] * gd;
        Gam[mm][k][l] = G.Gu[mm][k][l] - 0.5 * ichi * dk;
      }
  double E[3][3], DK[3][3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double kk = 0.0;
      for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) kk += Kij[i][k] * gamu[k][l] * Kij[l][j];
      E[i][j] = G.R[i][j] + K * Kij[i][j] - kk;
    }
  for (int k = 0; k < 3; ++k)
    for (int l = 0; l < 3; ++l)
      for (int j = 0; j < 3; ++j) {
        double s = dKij[k][l][j];
        for (int mm = 0; mm < 3; ++mm) s -= Gam[mm][k][l] * Kij[mm][j] + Gam[mm][k][j] * Kij[l][mm];
        DK[k][l][j] = s;
      }
  const double sqrtg = sqrt(det3(gam));
  double Bt[3][3], B[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0.0;
      for (int mm = 0; mm < 3; ++mm)
        for (int k = 0; k < 3; ++k)
          for (int l = 0; l < 3; ++l) {
            /* Levi-Civita symbol [mkl] */
            double e = (double)((mm - k) * (k - l) * (l - mm)) / 2.0;
            if (e != 0.0) s += gam[i][mm] * e / sqrtg * DK[k][l][j];
          }
      Bt[i][j] = s;
    }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) B[i][j] = 0.5 * (Bt[i][j] + Bt[j][i]);
  /* tetrad */
  double u[3][3] = {{x[0], x[1], x[2]},
                    {-x[1], x[0], 0.0},
                    {x[0] * x[2], x[1] * x[2], -(x[0] * x[0] + x[1] * x[1])}};
  double e[3][3]; /* e_r, e_ph, e_th */
  for (int a = 0; a < 3; ++a) {
    double v[3] = {u[a][0], u[a][1], u[a][2]};
    for (int b = 0; b < a; ++b) {
      double d = 0.0;
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) d += gam[i][j] * e[b][i] * v[j];
      for (int i = 0; i < 3; ++i) v[i] -= d * e[b][i];
    }
    double nn = 0.0;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) nn += gam[i][j] * v[i] * v[j];
    for (int i = 0; i < 3; ++i) e[a][i] = v[i] / sqrt(nn);
  }
  const double *ph = e[1], *th = e[2];
  double Ett = 0, Epp = 0, Etp = 0, Btt = 0, Bpp = 0, Btp = 0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      Ett += E[i][j] * th[i] * th[j];
      Epp += E[i][j] * ph[i] * ph[j];
      Etp += E[i][j] * th[i] * ph[j];
      Btt += B[i][j] * th[i] * th[j];
      Bpp += B[i][j] * ph[i] * ph[j];
      Btp += B[i][j] * th[i] * ph[j];
    }
  /* mb^i mb^j = (th th - ph ph - i (th ph + ph th)) / 2 */
  out[0] = 0.5 * (Ett - Epp) - Btp;
  out[1] = -Etp - 0.5 * (Btt - Bpp);
}

/* Psi4 at every interior cell: out holds, per block, the real part and then
 * the imaginary part over the block's storage cells; other cells get 0.
 * `u` must have its ghosts filled. */
void orc_psi4(const orc_mesh *m, const double *u, double *out) {
  long off = 0;
  for (int b = 0; b < m->nblocks; ++b) {
    long e0 = ext(m, b, 0), e1 = ext(m, b, 1), e2 = ext(m, b, 2);
    long S = e0 * e1 * e2;
    long st[3] = {1, e0, e0 * e1};
    const double *base = u + blk_offset(m, b);
#pragma omp parallel for schedule(static)
    for (long k = 0; k < e2; ++k)
      for (long j = 0; j < e1; ++j)
        for (long i = 0; i < e0; ++i) {
          long cidx = (k * e1 + j) * e0 + i;
          double v[2] = {0.0, 0.0};
          if (is_interior(m, b, (int)i, (int)j, (int)k)) {
            double x[3];
            cell_centre(m, b, (int)i, (int)j, (int)k, x);
            psi4_point(m, base + cidx, S, st, m->h[b], x, v);
          }
          out[off + cidx] = v[0];
          out[off + S + cidx] = v[1];
        }
    off += 2 * S;
  }
}

void orc_constraints(const orc_mesh *m, const double *u, double r_mask, double *per_cell, double norms[6]) {
  double sH = 0, sM = 0, sV = 0, mH = 0, sHm = 0, sMm = 0, sVm = 0, mM = 0;
  long pc_off = 0;
  for (int b = 0; b < m->nblocks; ++b) {
    long e0 = ext(m, b, 0), e1 = ext(m, b, 1), e2 = ext(m, b, 2);
    long S = e0 * e1 * e2;
    long st[3] = {1, e0, e0 * e1};
    const double *base = u + blk_offset(m, b);
    double h = m->h[b], vol = h * h * h;
    for (long k = 0; k < e2; ++k)
      for (long j = 0; j < e1; ++j)
        for (long i = 0; i < e0; ++i) {
          long cidx = (k * e1 + j) * e0 + i;
          if (!is_interior(m, b, (int)i, (int)j, (int)k)) {
            if (per_cell)
              for (int q = 0; q < 4; ++q) per_cell[pc_off + q * S + cidx] = 0.0;
            continue;
          }
          point_data P;
          geometry G;
          gather_point(m, base + cidx, S, st, h, &P, 1);
          compute_geometry(m, &P, &G);
          double H = G.Rs + 2.0 / 3.0 * G.K * G.K - G.AA;
          /* d_k gt^ij = - gt^ia gt^jb d_k gt_ab */
          double dgi[3][3][3];
          for (int kk = 0; kk < 3; ++kk)
            for (int a = 0; a < 3; ++a)
              for (int c2 = 0; c2 < 3; ++c2) {
                double s = 0.0;
                for (int p = 0; p < 3; ++p)
                  for (int q = 0; q < 3; ++q) s -= G.gi[a][p] * G.gi[c2][q] * P.dg[kk][p][q];
                dgi[kk][a][c2] = s;
              }
          double M[3];
          double dK[3];
          for (int kk = 0; kk < 3; ++kk) dK[kk] = P.dKhat[kk] + 2.0 * P.dTheta[kk];
          for (int a = 0; a < 3; ++a) {
            double s = 0.0;
            /* d_j At^aj by the product rule */
            for (int jj = 0; jj < 3; ++jj)
              for (int p = 0; p < 3; ++p)
                for (int q = 0; q < 3; ++q)
                  s += dgi[jj][a][p] * G.gi[jj][q] * P.A[p][q] + G.gi[a][p] * dgi[jj][jj][q] * P.A[p][q] +
                       G.gi[a][p] * G.gi[jj][q] * P.dA[jj][p][q];
            for (int jj = 0; jj < 3; ++jj)
              for (int kk = 0; kk < 3; ++kk) s += G.Gu[a][jj][kk] * G.Au[jj][kk];
            for (int jj = 0; jj < 3; ++jj) s -= 1.5 / G.chig * G.Au[a][jj] * P.dchi[jj];
            for (int jj = 0; jj < 3; ++jj) s -= 2.0 / 3.0 * G.gi[a][jj] * dK[jj];
            M[a] = s;
          }
          double M2 = M[0] * M[0] + M[1] * M[1] + M[2] * M[2];
          sH += H * H * vol;
          sM += M2 * vol;
          sV += vol;
          if (fabs(H) > mH) mH = fabs(H);
          if (sqrt(M2) > mM) mM = sqrt(M2);
          double x[3];
          cell_centre(m, b, (int)i, (int)j, (int)k, x);
          double r = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
          if (r > r_mask) {
            sHm += H * H * vol;
            sMm += M2 * vol;
            sVm += vol;
          }
          if (per_cell) {
            per_cell[pc_off + cidx] = H;
            for (int q = 0; q < 3; ++q) per_cell[pc_off + (q + 1) * S + cidx] = M[q];
          }
        }
    pc_off += 4 * S;
  }
  norms[0] = sqrt(sH / sV);
  norms[1] = sqrt(sM / sV);
  norms[2] = mH;
  norms[3] = sVm > 0 ? sqrt(sHm / sVm) : 0.0;
  norms[4] = sVm > 0 ? sqrt(sMm / sVm) : 0.0;
  norms[5] = mM;
}

/* ------------------------------------------------------------------ */
/* analytic initial data on every storage cell (ghosts included)       */
/* ------------------------------------------------------------------ */

/* kind 0: flat space.
 * kind 1: gauge wave along x, par = {A, d, t}:  H = 1 - A sin(2 pi (x - t)/d),
 *         ds^2 = -H dt^2 + H dx^2 + dy^2 + dz^2, zero shift.
 * kind 2: linear TT wave along x, par = {A, d, t}: gamma_yy = 1 + a,
 *         gamma_zz = 1 - a, a = A sin(2 pi (x - t)/d), K_ij = -1/2 d_t gamma_ij,
 *         alpha = 1, zero shift.
 * kind 3: Schwarzschild in isotropic coordinates at the origin,
 *         par = {M, lapse_kind}: psi = 1 + M/(2r), chi = psi^-4, gt = delta,
 *         At = Khat = Theta = Gam = 0, zero shift; alpha = psi^-2
 *         (lapse_kind 0, "pre-collapsed") or (1 - M/2r)/(1 + M/2r)
 *         (lapse_kind 1, the static lapse).
 * kind 4: Brill-Lindquist punctures, par = {np, m_1, x_1, y_1, z_1, ...}:
 *         psi = 1 + sum m_a / (2 r_a), alpha = psi^-2, otherwise as kind 3. */
static void id_point(int kind, const double *par, const double x[3], double v[NF]) {
  for (int f = 0; f < NF; ++f) v[f] = 0.0;
  v[F_CHI] = 1.0;
  v[F_GXX] = v[F_GYY] = v[F_GZZ] = 1.0;
  v[F_ALPHA] = 1.0;
  const double pi = 3.14159265358979323846;
  if (kind == 1) {
    double A = par[0], d = par[1], t = par[2];
    double ph = 2.0 * pi * (x[0] - t) / d;
    double H = 1.0 - A * sin(ph);
    double Kxx = -pi * A / d * cos(ph) / sqrt(H);
    double K = Kxx / H;
    double chi = pow(H, -1.0 / 3.0);
    v[F_CHI] = chi;
    v[F_GXX] = pow(H, 2.0 / 3.0);
    v[F_GYY] = chi;
    v[F_GZZ] = chi;
    v[F_KHAT] = K;
    v[F_AXX] = 2.0 / 3.0 * chi * Kxx;
    v[F_AYY] = -chi * K / 3.0;
    v[F_AZZ] = -chi * K / 3.0;
    v[F_GAMX] = -4.0 * pi * A / (3.0 * d) * cos(ph) * pow(H, -5.0 / 3.0);
    v[F_ALPHA] = sqrt(H);
  } else if (kind == 2) {
    double A = par[0], d = par[1], t = par[2];
    double ph = 2.0 * pi * (x[0] - t) / d;
    double a = A * sin(ph);
    double da = 2.0 * pi / d * A * cos(ph);  /* d_x a = -d_t a */
    double gyy = 1.0 + a, gzz = 1.0 - a;
    double Kyy = 0.5 * da, Kzz = -0.5 * da; /* -1/2 d_t gamma */
    double K = Kyy / gyy + Kzz / gzz;
    double chi = pow(gyy * gzz, -1.0 / 3.0);
    v[F_CHI] = chi;
    v[F_GXX] = chi;
    v[F_GYY] = chi * gyy;
    v[F_GZZ] = chi * gzz;
    v[F_KHAT] = K;
    v[F_AXX] = chi * (0.0 - K / 3.0);
    v[F_AYY] = chi * (Kyy - gyy * K / 3.0);
    v[F_AZZ] = chi * (Kzz - gzz * K / 3.0);
    /* Gam^x = -d_x gt^xx, gt^xx = 1/chi = (1 - a^2)^(1/3) */
    v[F_GAMX] = 2.0 / 3.0 * a * da * pow(1.0 - a * a, -2.0 / 3.0);
  } else if (kind == 3 || kind == 4) {
    double psi = 1.0;
    double M = 0.0;
    if (kind == 3) {
      M = par[0];
      double r = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
      psi += M / (2.0 * r);
      if ((int)par[1] == 1)
        v[F_ALPHA] = (1.0 - M / (2.0 * r)) / (1.0 + M / (2.0 * r));
      else
        v[F_ALPHA] = 1.0 / (psi * psi);
    } else {
      int np = (int)par[0];
      for (int a = 0; a < np; ++a) {
        const double *q = par + 1 + 4 * a;
        double dx = x[0] - q[1], dy = x[1] - q[2], dz = x[2] - q[3];
        psi += q[0] / (2.0 * sqrt(dx * dx + dy * dy + dz * dz));
      }
      v[F_ALPHA] = 1.0 / (psi * psi);
    }
    v[F_CHI] = 1.0 / (psi * psi * psi * psi);
  }
}

void orc_initial_data(const orc_mesh *m, double *u, int kind, const double *par) {
  for (int b = 0; b < m->nblocks; ++b) {
    long e0 = ext(m, b, 0), e1 = ext(m, b, 1), e2 = ext(m, b, 2);
    long S = e0 * e1 * e2;
    double *base = u + blk_offset(m, b);
    for (long k = 0; k < e2; ++k)
      for (long j = 0; j < e1; ++j)
        for (long i = 0; i < e0; ++i) {
          double x[3], v[NF];
          cell_centre(m, b, (int)i, (int)j, (int)k, x);
          id_point(kind, par, x, v);
          long cidx = (k * e1 + j) * e0 + i;
          for (int f = 0; f < NF; ++f) base[f * S + cidx] = v[f];
        }
  }
}

int orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* diagnostics beside the step (Sec. 3.2 refinement criteria, Sec. 3.3  */
/* puncture trackers)                                                   */
/* ------------------------------------------------------------------ */

/* Refinement indicators of every block (Sec. 3.2): over the block's
 * interior cells, chi_min[b] = min chi (the chi-min criterion) and
 * dchi_max[b] = max |grad chi| (the d-chi criterion), the gradient by the
 * centred first-derivative stencil of order m->order (reading R17).  Ghost
 * cells must be filled. */
void orc_block_indicators(const orc_mesh *m, const double *u, double *chi_min, double *dchi_max) {
  for (int b = 0; b < m->nblocks; ++b) {
    const long e0 = ext(m, b, 0), e1 = ext(m, b, 1);
    const long st[3] = {1, e0, e0 * e1};
    const double *chi = u + blk_offset(m, b) + (long)F_CHI * e0 * e1 * ext(m, b, 2);
    const int g = m->ghosts;
    double mn = INFINITY, mx = 0.0;
    for (int k = g; k < g + m->n[3 * b + 2]; ++k)
      for (int j = g; j < g + m->n[3 * b + 1]; ++j)
        for (int i = g; i < g + m->n[3 * b]; ++i) {
          const double *p = chi + ((long)k * e1 + j) * e0 + i;
          if (*p < mn) mn = *p;
          double s = 0.0;
          for (int d = 0; d < 3; ++d) {
            const double q = d1(p, st[d], m->order, m->h[b]);
            s += q * q;
          }
          const double a = sqrt(s);
          if (a > mx) mx = a;
        }
    chi_min[b] = mn;
    dchi_max[b] = mx;
  }
}

/* The first block (in block order) whose closed box [lo, lo + n h] contains
 * x, within 1e-12 h; -1 if none. */
static int block_containing(const orc_mesh *m, const double x[3]) {
  for (int b = 0; b < m->nblocks; ++b) {
    int in = 1;
    for (int d = 0; d < 3; ++d) {
      const double t = (x[d] - m->lo[3 * b + d]) / m->h[b];
      in &= t >= -1e-12 && t <= m->n[3 * b + d] + 1e-12;
    }
    if (in) return b;
  }
  return -1;
}

/* Puncture tracker (Sec. 3.3): a puncture moves with dx/dt = -beta(x).  One
 * forward-Euler step x <- x - dt beta(x) per call (reading R18), beta from
 * block_containing(x) by 4-point Lagrange interpolation per axis (3D tensor
 * product) over the cell centres i0 .. i0 + 3, i0 = floor((x - lo)/h - 1/2)
 * - 1.  Ghost cells must be filled.  beta_out (nullable): the 3 components
 * per puncture.  Returns 0, or -1 if a puncture lies in no block. */
int orc_track_punctures(const orc_mesh *m, const double *u, int np, double *xyz, double dt,
                        double *beta_out) {
  for (int q = 0; q < np; ++q) {
    double x[3] = {xyz[3 * q], xyz[3 * q + 1], xyz[3 * q + 2]};
    if (m->periodic) wrap(m, x);
    const int b = block_containing(m, x);
    if (b < 0) return -1;
    const long e0 = ext(m, b, 0), e1 = ext(m, b, 1), S = e0 * e1 * ext(m, b, 2);
    const double h = m->h[b];
    long s0[3];
    double w[3][4];
    for (int d = 0; d < 3; ++d) {
      const double lo = m->lo[3 * b + d];
      const long i0 = (long)floor((x[d] - lo) / h - 0.5) - 1;
      s0[d] = i0 + m->ghosts;
      double xs[4];
      for (int a = 0; a < 4; ++a) xs[a] = lo + (i0 + a + 0.5) * h;
      for (int a = 0; a < 4; ++a) w[d][a] = lagrange(xs, 4, a, x[d]);
    }
    const double *base = u + blk_offset(m, b);
    double beta[3];
    for (int c = 0; c < 3; ++c) {
      const double *f = base + (long)(F_BETAX + c) * S;
      double v = 0.0;
      for (int kz = 0; kz < 4; ++kz)
        for (int jy = 0; jy < 4; ++jy)
          for (int ix = 0; ix < 4; ++ix)
            v += w[2][kz] * w[1][jy] * w[0][ix] * f[((s0[2] + kz) * e1 + s0[1] + jy) * e0 + s0[0] + ix];
      beta[c] = v;
    }
    for (int d = 0; d < 3; ++d) {
      xyz[3 * q + d] -= dt * beta[d];
      if (beta_out) beta_out[3 * q + d] = beta[d];
    }
  }
  return 0;
}
