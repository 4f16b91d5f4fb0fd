/*
 * pff_oracle.c -- plain FP64 CPU oracle for the matrix-free phase-field
 * fracture step (arxiv 2606.23458).  TEST INFRASTRUCTURE ONLY: the tests,
 * the smoke check and the bench's CPU-baseline leg call it; the CUDA path
 * never does.  It shares no code with the CUDA library.
 *
 * Everything is written as the paper states it, one element or one node at
 * a time, in element-id order, with no blocking or fusion:
 *   - P1 geometry, Eq. (grad_phi) of Sec. 2.3; lumped mass and CFL step of
 *     the velocity-Verlet paragraph (Sec. 2.3);
 *   - energy splits: Eq. (spectral_split) and Eq. (amor_split), degradation
 *     g(d) = (1-d)^2 + eta (Sec. 2.1); plane-strain Lame constants (Sec. 2.1,
 *     "Plane assumptions");
 *   - internal force by gather / element contraction / scatter (Sec. 2.3);
 *   - velocity Verlet, Eqs. (vv_u), (vv_a), (vv_v);
 *   - history H = max(H, psi+) and the staggered order (Sec. 2.2);
 *   - AT2 damage equation, Eq. (damage_pde_at2), Jacobi-preconditioned CG and
 *     post-clamp (Sec. 2.4); AT1 inequality, Eq. (damage_pde_at1), by a
 *     projected CG with an active set (Sec. 2.4); consistent damage mass
 *     M^e_ij = A_e (1 + delta_ij) / 12 (Sec. 2.4);
 *   - smooth traction ramp, Eq. (smooth_traction_ramp) (Sec. 3);
 *   - energies per unit thickness, Eq. (total_energy) and Sec. 3.1;
 *   - implicit differentiation of the damage solve, Eqs.
 *     (implicit_forward_linear_system), (implicit_adjoint_linear_system),
 *     (implicit_gc_l0_element_term), with active-set masking (Sec. 4.2), and
 *     the reverse of the explicit step for dL/dGc.
 *
 * Readings taken where the paper is silent (each is listed in the design
 * notes): H lives per element; g is evaluated at the element-mean damage;
 * the notch is a Dirichlet set d = 1; CG stops on the unpreconditioned
 * residual ||r||_2 <= tol ||b_eff||_2 with warm start x0 = d_n; eta only
 * enters the stress, not the damage operator; AT2 is clamped to [d_n, 1];
 * AT1 bounds are [d_n, 1].
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_ERR_ARG 1
#define OR_ERR_MESH 2
#define OR_ERR_NOT_CONVERGED 5

enum { OR_AT1 = 1, OR_AT2 = 2 };
enum { OR_SPECTRAL = 0, OR_AMOR = 1, OR_ISO = 2 };
enum { OR_PLANE_STRAIN = 0, OR_PLANE_STRESS = 1 };

typedef struct {
  double E, nu, rho, Gc, l0, eta;
  int32_t model, split, plane, pad;
} or_material;

typedef struct {
  int64_t N, Ne;
  double *x, *y;        /* node coordinates */
  int32_t *t;           /* Ne x 3 connectivity */
  uint8_t *notch;       /* N: Dirichlet damage set (d = 1) */
  double *area;         /* Ne */
  double *grad;         /* Ne x 3 x 2: (dphi_a/dx, dphi_a/dy) */
  double *fext;         /* N x 2 nodal traction load at full scale */
  double hmin;          /* min over elements of the incircle diameter 4A/P */
  double *gcf;          /* Ne: per-element toughness Gc_e (Secs. 4.2, 7: the
                           field-valued inverse), NULL: the material's Gc */
} or_mesh;

/* ------------------------------------------------------------------ mesh */

/* Builds the P1 geometry of Eq. (grad_phi).  Returns NULL and sets *bad to
 * the first element with A_e <= 0 when the mesh is inverted/degenerate. */
or_mesh *or_mesh_create(int64_t N, const double *xy, int64_t Ne,
                        const int32_t *tri, const uint8_t *notch, int64_t M,
                        const int32_t *tedges, const double *tvec,
                        int64_t *bad) {
  *bad = -1;
  if (N <= 0 || Ne <= 0) return NULL;
  for (int64_t e = 0; e < 3 * Ne; ++e)
    if (tri[e] < 0 || tri[e] >= N) { *bad = e / 3; return NULL; }
  or_mesh *m = (or_mesh *)calloc(1, sizeof(or_mesh));
  m->N = N; m->Ne = Ne;
  m->x = (double *)malloc(N * sizeof(double));
  m->y = (double *)malloc(N * sizeof(double));
  m->t = (int32_t *)malloc(3 * Ne * sizeof(int32_t));
  m->notch = (uint8_t *)calloc(N, 1);
  m->area = (double *)malloc(Ne * sizeof(double));
  m->grad = (double *)malloc(6 * Ne * sizeof(double));
  m->fext = (double *)calloc(2 * N, sizeof(double));
  for (int64_t i = 0; i < N; ++i) { m->x[i] = xy[2 * i]; m->y[i] = xy[2 * i + 1]; }
  memcpy(m->t, tri, 3 * Ne * sizeof(int32_t));
  if (notch) memcpy(m->notch, notch, N);
  m->hmin = INFINITY;
  for (int64_t e = 0; e < Ne; ++e) {
    int32_t n1 = tri[3 * e], n2 = tri[3 * e + 1], n3 = tri[3 * e + 2];
    double x1 = m->x[n1], y1 = m->y[n1], x2 = m->x[n2], y2 = m->y[n2];
    double x3 = m->x[n3], y3 = m->y[n3];
    double A = 0.5 * ((x2 - x1) * (y3 - y1) - (x3 - x1) * (y2 - y1));
    if (!(A > 0.0)) {
      *bad = e;
      free(m->x); free(m->y); free(m->t); free(m->notch); free(m->area);
      free(m->grad); free(m->fext); free(m);
      return NULL;
    }
    m->area[e] = A;
    double s = 1.0 / (2.0 * A);
    double *g = m->grad + 6 * e;
    g[0] = s * (y2 - y3); g[1] = s * (x3 - x2);
    g[2] = s * (y3 - y1); g[3] = s * (x1 - x3);
    g[4] = s * (y1 - y2); g[5] = s * (x2 - x1);
    double P = hypot(x2 - x1, y2 - y1) + hypot(x3 - x2, y3 - y2) +
               hypot(x1 - x3, y1 - y3);
    double hin = 4.0 * A / P;
    if (hin < m->hmin) m->hmin = hin;
  }
  /* Consistent P1 load of a constant traction on a boundary edge: half the
   * edge force to each end node, accumulated in edge order. */
  for (int64_t k = 0; k < M; ++k) {
    int32_t i = tedges[2 * k], j = tedges[2 * k + 1];
    double L = hypot(m->x[j] - m->x[i], m->y[j] - m->y[i]);
    for (int c = 0; c < 2; ++c) {
      m->fext[2 * i + c] += 0.5 * L * tvec[2 * k + c];
      m->fext[2 * j + c] += 0.5 * L * tvec[2 * k + c];
    }
  }
  return m;
}

void or_mesh_free(or_mesh *m) {
  if (!m) return;
  free(m->x); free(m->y); free(m->t); free(m->notch); free(m->area);
  free(m->grad); free(m->fext); free(m->gcf); free(m);
}

/* Per-element toughness field (gc: Ne values, copied; NULL restores the
 * material's uniform Gc). */
void or_mesh_set_gc_field(or_mesh *m, const double *gc) {
  free(m->gcf);
  m->gcf = NULL;
  if (!gc) return;
  m->gcf = (double *)malloc(m->Ne * sizeof(double));
  memcpy(m->gcf, gc, m->Ne * sizeof(double));
}

/* Toughness of element e. */
static double elem_gc(const or_mesh *m, const or_material *mt, int64_t e) {
  return m->gcf ? m->gcf[e] : mt->Gc;
}

void or_mesh_geometry(const or_mesh *m, double *area, double *grad,
                      double *fext, double *hmin) {
  if (area) memcpy(area, m->area, m->Ne * sizeof(double));
  if (grad) memcpy(grad, m->grad, 6 * m->Ne * sizeof(double));
  if (fext) memcpy(fext, m->fext, 2 * m->N * sizeof(double));
  if (hmin) *hmin = m->hmin;
}

/* Lumped mass m_i = rho * sum_{e containing i} A_e / 3, element order. */
void or_lumped_mass(const or_mesh *m, double rho, double *mass) {
  memset(mass, 0, m->N * sizeof(double));
  for (int64_t e = 0; e < m->Ne; ++e)
    for (int a = 0; a < 3; ++a) mass[m->t[3 * e + a]] += rho * m->area[e] / 3.0;
}

/* Node-to-element incidence: for node i, entries ptr[i]..ptr[i+1]-1 hold
 * (e << 2) | slot for every element e containing i at local slot `slot`,
 * in ascending element id. */
void or_csr(const or_mesh *m, int32_t *ptr, int32_t *ent) {
  int64_t N = m->N, Ne = m->Ne;
  int32_t *fill = (int32_t *)calloc(N, sizeof(int32_t));
  memset(ptr, 0, (N + 1) * sizeof(int32_t));
  for (int64_t e = 0; e < Ne; ++e)
    for (int a = 0; a < 3; ++a) ptr[m->t[3 * e + a] + 1] += 1;
  for (int64_t i = 0; i < N; ++i) ptr[i + 1] += ptr[i];
  for (int64_t e = 0; e < Ne; ++e)
    for (int a = 0; a < 3; ++a) {
      int32_t i = m->t[3 * e + a];
      ent[ptr[i] + fill[i]++] = (int32_t)((e << 2) | a);
    }
  free(fill);
}

/* Greedy element colouring in element-id order: each element takes the
 * smallest colour not used by an earlier element that shares a node.
 * Returns the number of colours. */
int or_colour(const or_mesh *m, uint8_t *colour) {
  int64_t N = m->N, Ne = m->Ne;
  int32_t *ptr = (int32_t *)malloc((N + 1) * sizeof(int32_t));
  int32_t *ent = (int32_t *)malloc(3 * Ne * sizeof(int32_t));
  or_csr(m, ptr, ent);
  int ncol = 0;
  for (int64_t e = 0; e < Ne; ++e) {
    int used[256] = {0};
    for (int a = 0; a < 3; ++a) {
      int32_t i = m->t[3 * e + a];
      for (int32_t k = ptr[i]; k < ptr[i + 1]; ++k) {
        int64_t f = ent[k] >> 2;
        if (f < e) used[colour[f]] = 1;
      }
    }
    int c = 0;
    while (used[c]) ++c;
    colour[e] = (uint8_t)c;
    if (c + 1 > ncol) ncol = c + 1;
  }
  free(ptr); free(ent);
  return ncol;
}

/* ------------------------------------------------------------- material */

typedef struct { double lam, mu, K, cz; } or_lame;

/* Sec. 2.1, "Plane assumptions": the first Lame parameter of the plane
 * model, lambda_PE = E nu / ((1+nu)(1-2nu)) (plane strain) or
 * lambda_PS = E nu / (1 - nu^2) (plane stress); mu = E / (2(1+nu)); the
 * 3-D bulk modulus K = E / (3(1-2nu)) in both; cz = nu / (1 - nu) under
 * plane stress (e_zz = -cz tr_2D enters the 3-D trace of the
 * volumetric-deviatoric split), 0 under plane strain (e_zz = 0). */
static or_lame lame_of(const or_material *mt) {
  or_lame L;
  const int ps = mt->plane == OR_PLANE_STRESS;
  L.lam = ps ? mt->E * mt->nu / (1.0 - mt->nu * mt->nu)
             : mt->E * mt->nu / ((1.0 + mt->nu) * (1.0 - 2.0 * mt->nu));
  L.mu = mt->E / (2.0 * (1.0 + mt->nu));
  L.K = mt->E / (3.0 * (1.0 - 2.0 * mt->nu));
  L.cz = ps ? mt->nu / (1.0 - mt->nu) : 0.0;
  return L;
}

/* Stable step dt = cfl * h_min / c_p with c_p = sqrt((lambda + 2 mu)/rho). */
double or_stable_dt(const or_mesh *m, const or_material *mt, double cfl) {
  or_lame L = lame_of(mt);
  double cp = sqrt((L.lam + 2.0 * L.mu) / mt->rho);
  return cfl * m->hmin / cp;
}

static double pos(double x) { return x > 0.0 ? x : 0.0; }
static double neg(double x) { return x < 0.0 ? x : 0.0; }

/* Constitutive update at one point.  e = (exx, eyy, exy) tensor components.
 * Outputs sp = sigma+, sm = sigma- (tensor components) and psi+/psi-. */
static void split_point(const or_material *mt, const double e[3], double sp[3],
                        double sm[3], double *psip, double *psim) {
  or_lame L = lame_of(mt);
  double tr = e[0] + e[1];
  if (mt->split == OR_SPECTRAL) {
    /* Eq. (spectral_split): principal strains of the in-plane tensor (the
     * plane-strain e_zz = 0 adds nothing), projectors P1, P2 onto them. */
    double half = 0.5 * (e[0] - e[1]);
    double R = sqrt(half * half + e[2] * e[2]);
    double e1 = 0.5 * tr + R, e2 = 0.5 * tr - R;
    double P1[3], P2[3];
    if (R > 0.0) {
      P1[0] = 0.5 + half / (2.0 * R);
      P1[1] = 0.5 - half / (2.0 * R);
      P1[2] = e[2] / (2.0 * R);
    } else {
      P1[0] = 1.0; P1[1] = 1.0; P1[2] = 0.0;
    }
    P2[0] = 1.0 - P1[0]; P2[1] = 1.0 - P1[1]; P2[2] = -P1[2];
    double ep[3];
    /* R = 0: one double eigenvalue, P1 = I carries it and P2 = 0. */
    for (int c = 0; c < 3; ++c) ep[c] = pos(e1) * P1[c] + pos(e2) * P2[c];
    sp[0] = L.lam * pos(tr) + 2.0 * L.mu * ep[0];
    sp[1] = L.lam * pos(tr) + 2.0 * L.mu * ep[1];
    sp[2] = 2.0 * L.mu * ep[2];
    sm[0] = L.lam * neg(tr) + 2.0 * L.mu * (e[0] - ep[0]);
    sm[1] = L.lam * neg(tr) + 2.0 * L.mu * (e[1] - ep[1]);
    sm[2] = 2.0 * L.mu * (e[2] - ep[2]);
    *psip = 0.5 * L.lam * pos(tr) * pos(tr) + L.mu * (pos(e1) * pos(e1) + pos(e2) * pos(e2));
    *psim = 0.5 * L.lam * neg(tr) * neg(tr) + L.mu * (neg(e1) * neg(e1) + neg(e2) * neg(e2));
  } else if (mt->split == OR_AMOR) {
    /* Eq. (amor_split) on the 3-D strain (e_xx, e_yy, e_xy; e_zz) with
     * e_zz = -cz tr (0 in plane strain): tr3 = tr + e_zz,
     * e_dev:e_dev = e:e + e_zz^2 - tr3^2/3.  The in-plane stresses are the
     * derivatives of psi+- with respect to the in-plane strain, e_zz
     * following it (d e_zz / d e_xx = d e_zz / d e_yy = -cz). */
    double ez = -L.cz * tr, tr3 = tr + ez, f = 1.0 - L.cz;
    double ee = e[0] * e[0] + e[1] * e[1] + 2.0 * e[2] * e[2] + ez * ez;
    double dz = L.cz * ez;  /* e_zz's share of d(e:e)/2 d e_xx, sign included */
    sp[0] = L.K * pos(tr3) * f + 2.0 * L.mu * (e[0] - dz - f * tr3 / 3.0);
    sp[1] = L.K * pos(tr3) * f + 2.0 * L.mu * (e[1] - dz - f * tr3 / 3.0);
    sp[2] = 2.0 * L.mu * e[2];
    sm[0] = L.K * neg(tr3) * f;
    sm[1] = L.K * neg(tr3) * f;
    sm[2] = 0.0;
    *psip = 0.5 * L.K * pos(tr3) * pos(tr3) + L.mu * (ee - tr3 * tr3 / 3.0);
    *psim = 0.5 * L.K * neg(tr3) * neg(tr3);
  } else {
    /* isotropic: psi+ = psi, psi- = 0 (Sec. 2.1). */
    double ee = e[0] * e[0] + e[1] * e[1] + 2.0 * e[2] * e[2];
    sp[0] = L.lam * tr + 2.0 * L.mu * e[0];
    sp[1] = L.lam * tr + 2.0 * L.mu * e[1];
    sp[2] = 2.0 * L.mu * e[2];
    sm[0] = sm[1] = sm[2] = 0.0;
    *psip = 0.5 * L.lam * tr * tr + L.mu * ee;
    *psim = 0.0;
  }
}

static double degr(const or_material *mt, double d) {
  return (1.0 - d) * (1.0 - d) + mt->eta;
}

/* Exposed for the pins: sigma = g(d) sigma+ + sigma-, psi = g psi+ + psi-. */
void or_constitutive(const or_material *mt, const double e[3], double dbar,
                     double sig[3], double sigp[3], double *psip, double *psim,
                     double *psi) {
  double sp[3], sm[3];
  split_point(mt, e, sp, sm, psip, psim);
  double g = degr(mt, dbar);
  for (int c = 0; c < 3; ++c) { sig[c] = g * sp[c] + sm[c]; if (sigp) sigp[c] = sp[c]; }
  *psi = g * (*psip) + (*psim);
}

/* Tangent action of the split: dsp = D sigma+[de], dsm = D sigma-[de].
 * Kinks use <x>+'(0) = 0; a double principal strain uses the limit ratio
 * H(e1) (Heaviside with H(0) = 0). */
static void split_tangent(const or_material *mt, const double e[3],
                          const double de[3], double dsp[3], double dsm[3]) {
  or_lame L = lame_of(mt);
  double tr = e[0] + e[1], dtr = de[0] + de[1];
  double Htr = tr > 0.0 ? 1.0 : 0.0;
  if (mt->split == OR_SPECTRAL) {
    double half = 0.5 * (e[0] - e[1]);
    double R = sqrt(half * half + e[2] * e[2]);
    double e1 = 0.5 * tr + R, e2 = 0.5 * tr - R;
    /* 2x2 symmetric matrices as full arrays [xx xy; xy yy]. */
    double P1[2][2], P2[2][2], D[2][2];
    if (R > 0.0) {
      P1[0][0] = 0.5 + half / (2.0 * R); P1[1][1] = 0.5 - half / (2.0 * R);
      P1[0][1] = P1[1][0] = e[2] / (2.0 * R);
    } else {
      P1[0][0] = 1.0; P1[1][1] = 1.0; P1[0][1] = P1[1][0] = 0.0;
    }
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j) P2[i][j] = (i == j ? 1.0 : 0.0) - P1[i][j];
    D[0][0] = de[0]; D[1][1] = de[1]; D[0][1] = D[1][0] = de[2];
    double p1d = P1[0][0] * D[0][0] + P1[1][1] * D[1][1] + 2.0 * P1[0][1] * D[0][1];
    double p2d = P2[0][0] * D[0][0] + P2[1][1] * D[1][1] + 2.0 * P2[0][1] * D[0][1];
    double H1 = e1 > 0.0 ? 1.0 : 0.0, H2 = e2 > 0.0 ? 1.0 : 0.0;
    double theta = (R > 0.0) ? (pos(e1) - pos(e2)) / (e1 - e2) : H1;
    /* off = P1 D P2 + P2 D P1 */
    double off[2][2];
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j) {
        double s = 0.0;
        for (int k = 0; k < 2; ++k)
          for (int l = 0; l < 2; ++l)
            s += P1[i][k] * D[k][l] * P2[l][j] + P2[i][k] * D[k][l] * P1[l][j];
        off[i][j] = s;
      }
    double dep[2][2];
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j) {
        if (R > 0.0)
          dep[i][j] = H1 * p1d * P1[i][j] + H2 * p2d * P2[i][j] + theta * off[i][j];
        else
          dep[i][j] = H1 * D[i][j];
      }
    dsp[0] = L.lam * Htr * dtr + 2.0 * L.mu * dep[0][0];
    dsp[1] = L.lam * Htr * dtr + 2.0 * L.mu * dep[1][1];
    dsp[2] = 2.0 * L.mu * dep[0][1];
    dsm[0] = L.lam * (1.0 - Htr) * dtr + 2.0 * L.mu * (de[0] - dep[0][0]);
    dsm[1] = L.lam * (1.0 - Htr) * dtr + 2.0 * L.mu * (de[1] - dep[1][1]);
    dsm[2] = 2.0 * L.mu * (de[2] - dep[0][1]);
  } else if (mt->split == OR_AMOR) {
    /* derivative of the stresses above: tr3 = f tr, e_zz = -cz tr */
    double f = 1.0 - L.cz;
    double H3 = f * tr > 0.0 ? 1.0 : 0.0;
    double dlin = (L.cz * L.cz - f * f / 3.0) * dtr;  /* -cz d e_zz - f d tr3 / 3 */
    dsp[0] = L.K * H3 * f * f * dtr + 2.0 * L.mu * (de[0] + dlin);
    dsp[1] = L.K * H3 * f * f * dtr + 2.0 * L.mu * (de[1] + dlin);
    dsp[2] = 2.0 * L.mu * de[2];
    dsm[0] = L.K * (1.0 - H3) * f * f * dtr;
    dsm[1] = L.K * (1.0 - H3) * f * f * dtr;
    dsm[2] = 0.0;
  } else {
    dsp[0] = L.lam * dtr + 2.0 * L.mu * de[0];
    dsp[1] = L.lam * dtr + 2.0 * L.mu * de[1];
    dsp[2] = 2.0 * L.mu * de[2];
    dsm[0] = dsm[1] = dsm[2] = 0.0;
  }
}

void or_constitutive_tangent(const or_material *mt, const double e[3],
                             double dbar, const double de[3], double dsig[3]) {
  double dsp[3], dsm[3];
  split_tangent(mt, e, de, dsp, dsm);
  double g = degr(mt, dbar);
  for (int c = 0; c < 3; ++c) dsig[c] = g * dsp[c] + dsm[c];
}

/* Strain of element e from nodal displacement u (N x 2):
 * exx = sum dphi_a/dx u_xa, eyy = sum dphi_a/dy u_ya,
 * exy = 1/2 sum (dphi_a/dy u_xa + dphi_a/dx u_ya). */
static void elem_strain(const or_mesh *m, int64_t e, const double *u, double eps[3]) {
  const double *g = m->grad + 6 * e;
  eps[0] = eps[1] = eps[2] = 0.0;
  for (int a = 0; a < 3; ++a) {
    int32_t n = m->t[3 * e + a];
    eps[0] += g[2 * a] * u[2 * n];
    eps[1] += g[2 * a + 1] * u[2 * n + 1];
    eps[2] += 0.5 * (g[2 * a + 1] * u[2 * n] + g[2 * a] * u[2 * n + 1]);
  }
}

static double elem_dbar(const or_mesh *m, int64_t e, const double *d) {
  return (d[m->t[3 * e]] + d[m->t[3 * e + 1]] + d[m->t[3 * e + 2]]) / 3.0;
}

/* Internal force f = sum_e A_e B_e^T sigma_e, scattered in element order;
 * optionally returns psi+ per element (Sec. 2.3 gather-compute-scatter). */
void or_internal_force(const or_mesh *m, const or_material *mt, const double *u,
                       const double *d, double *f, double *psip_e) {
  memset(f, 0, 2 * m->N * sizeof(double));
  for (int64_t e = 0; e < m->Ne; ++e) {
    double eps[3], sig[3], sp[3], pp, pm, psi;
    elem_strain(m, e, u, eps);
    or_constitutive(mt, eps, elem_dbar(m, e, d), sig, sp, &pp, &pm, &psi);
    if (psip_e) psip_e[e] = pp;
    const double *g = m->grad + 6 * e;
    double A = m->area[e];
    for (int a = 0; a < 3; ++a) {
      int32_t n = m->t[3 * e + a];
      f[2 * n] += A * (sig[0] * g[2 * a] + sig[2] * g[2 * a + 1]);
      f[2 * n + 1] += A * (sig[2] * g[2 * a] + sig[1] * g[2 * a + 1]);
    }
  }
}

/* Smooth traction ramp, Eq. (smooth_traction_ramp). */
double or_ramp(double t, double tr) {
  if (t <= 0.0) return 0.0;
  if (t >= tr) return 1.0;
  return 0.5 * (1.0 - cos(3.14159265358979323846 * t / tr));
}

/* -------------------------------------------------------------- damage */

/* Coefficients of the damage operator A = sum_e [kappa_e K^e + c_e M^e] and
 * right-hand side b = sum_e w_e A_e / 3 per node, with the element's Gc:
 *   AT2, Eq. (damage_pde_at2): kappa = Gc l0, c_e = Gc/l0 + 2H_e, w_e = 2H_e;
 *   AT1, Eq. (damage_pde_at1): kappa = 3/4 Gc l0, c_e = 2H_e,
 *                              w_e = 2H_e - 3Gc/(8 l0). */
static double dmg_kappa(const or_mesh *m, const or_material *mt, int64_t e) {
  const double gc = elem_gc(m, mt, e);
  return mt->model == OR_AT1 ? 0.75 * gc * mt->l0 : gc * mt->l0;
}
static double dmg_c(const or_mesh *m, const or_material *mt, int64_t e, double H) {
  return mt->model == OR_AT1 ? 2.0 * H : elem_gc(m, mt, e) / mt->l0 + 2.0 * H;
}
static double dmg_w(const or_mesh *m, const or_material *mt, int64_t e, double H) {
  return mt->model == OR_AT1 ? 2.0 * H - 3.0 * elem_gc(m, mt, e) / (8.0 * mt->l0) : 2.0 * H;
}

/* q = A p over all nodes (no Dirichlet handling), element order:
 * q_a += kappa A_e sum_b (grad phi_a . grad phi_b) p_b
 *        + c_e A_e (1 + delta_ab)/12 p_b. */
void or_damage_apply(const or_mesh *m, const or_material *mt, const double *H,
                     const double *p, double *q) {
  memset(q, 0, m->N * sizeof(double));
  for (int64_t e = 0; e < m->Ne; ++e) {
    const double *g = m->grad + 6 * e;
    double kap = dmg_kappa(m, mt, e);
    double A = m->area[e], c = dmg_c(m, mt, e, H[e]);
    for (int a = 0; a < 3; ++a) {
      double s = 0.0;
      for (int b = 0; b < 3; ++b) {
        double Kab = A * (g[2 * a] * g[2 * b] + g[2 * a + 1] * g[2 * b + 1]);
        double Mab = A * (a == b ? 2.0 : 1.0) / 12.0;
        s += (kap * Kab + c * Mab) * p[m->t[3 * e + b]];
      }
      q[m->t[3 * e + a]] += s;
    }
  }
}

void or_damage_rhs(const or_mesh *m, const or_material *mt, const double *H,
                   double *b, double *diag) {
  memset(b, 0, m->N * sizeof(double));
  memset(diag, 0, m->N * sizeof(double));
  for (int64_t e = 0; e < m->Ne; ++e) {
    const double *g = m->grad + 6 * e;
    double kap = dmg_kappa(m, mt, e);
    double A = m->area[e], c = dmg_c(m, mt, e, H[e]), w = dmg_w(m, mt, e, H[e]);
    for (int a = 0; a < 3; ++a) {
      int32_t n = m->t[3 * e + a];
      b[n] += w * A / 3.0;
      diag[n] += kap * A * (g[2 * a] * g[2 * a] + g[2 * a + 1] * g[2 * a + 1]) +
                 c * A * 2.0 / 12.0;
    }
  }
}

static double dot_free(const or_mesh *m, const uint8_t *mask, const double *a,
                       const double *b) {
  double s = 0.0;
  for (int64_t i = 0; i < m->N; ++i)
    if (mask[i]) s += a[i] * b[i];
  return s;
}

typedef struct {
  double tol;
  int32_t max_it;
  int32_t max_restarts;
} or_solve_opts;

/* AT2 damage solve (Sec. 2.4): notch nodes are eliminated with x_D = 1,
 * Jacobi-PCG on the free nodes from x0 = d_prev, stop when
 * ||r||_2 <= tol * ||b - A 1_D||_2 (free rows), then
 * d = min(1, max(x, d_prev)), d_D = 1.
 * forced >= 0 runs exactly that many iterations (stopping early only on an
 * exactly zero p.q); *natural reports the count at which the stop test first
 * held (or -1).  x_out (nullable) receives the unclamped solution. */
static int solve_at2(const or_mesh *m, const or_material *mt, const double *H,
                     const double *dprev, double *dout, const or_solve_opts *o,
                     int forced, int *iters, int *natural, double *relres,
                     double *x_out) {
  int64_t N = m->N;
  double *b = malloc(N * sizeof(double)), *dg = malloc(N * sizeof(double));
  double *x = malloc(N * sizeof(double)), *r = malloc(N * sizeof(double));
  double *z = malloc(N * sizeof(double)), *p = malloc(N * sizeof(double));
  double *q = malloc(N * sizeof(double)), *oneD = malloc(N * sizeof(double));
  uint8_t *fr = malloc(N);
  int status = OR_OK;
  for (int64_t i = 0; i < N; ++i) fr[i] = m->notch[i] ? 0 : 1;
  or_damage_rhs(m, mt, H, b, dg);
  for (int64_t i = 0; i < N; ++i) oneD[i] = fr[i] ? 0.0 : 1.0;
  or_damage_apply(m, mt, H, oneD, q);
  double bn2 = 0.0;
  for (int64_t i = 0; i < N; ++i)
    if (fr[i]) bn2 += (b[i] - q[i]) * (b[i] - q[i]);
  double bn = sqrt(bn2);
  for (int64_t i = 0; i < N; ++i) x[i] = fr[i] ? dprev[i] : 1.0;
  or_damage_apply(m, mt, H, x, q);
  for (int64_t i = 0; i < N; ++i) r[i] = fr[i] ? b[i] - q[i] : 0.0;
  int k = 0;
  *natural = -1;
  double rr = dot_free(m, fr, r, r);
  if (bn == 0.0) {
    *relres = 0.0;
    *natural = 0;
  } else {
    if (sqrt(rr) <= o->tol * bn) *natural = 0;
    for (int64_t i = 0; i < N; ++i) { z[i] = fr[i] ? r[i] / dg[i] : 0.0; p[i] = z[i]; }
    double rho = dot_free(m, fr, r, z);
    for (;;) {
      if (forced >= 0) { if (k >= forced) break; }
      else if (sqrt(rr) <= o->tol * bn) break;
      if (k >= o->max_it) { status = OR_ERR_NOT_CONVERGED; break; }
      or_damage_apply(m, mt, H, p, q);
      for (int64_t i = 0; i < N; ++i) if (!fr[i]) q[i] = 0.0;
      double pq = dot_free(m, fr, p, q);
      if (pq == 0.0) break;
      double alpha = rho / pq;
      for (int64_t i = 0; i < N; ++i)
        if (fr[i]) { x[i] += alpha * p[i]; r[i] -= alpha * q[i]; }
      ++k;
      rr = dot_free(m, fr, r, r);
      if (*natural < 0 && sqrt(rr) <= o->tol * bn) *natural = k;
      for (int64_t i = 0; i < N; ++i) z[i] = fr[i] ? r[i] / dg[i] : 0.0;
      double rho_new = dot_free(m, fr, r, z);
      double beta = rho_new / rho;
      rho = rho_new;
      for (int64_t i = 0; i < N; ++i) p[i] = fr[i] ? z[i] + beta * p[i] : 0.0;
    }
    *relres = sqrt(rr) / bn;
  }
  *iters = k;
  if (x_out) memcpy(x_out, x, N * sizeof(double));
  for (int64_t i = 0; i < N; ++i) {
    double v = x[i] > dprev[i] ? x[i] : dprev[i];
    if (v > 1.0) v = 1.0;
    dout[i] = fr[i] ? v : 1.0;
  }
  free(b); free(dg); free(x); free(r); free(z); free(p); free(q); free(oneD); free(fr);
  return status;
}

/* AT1 damage solve (Sec. 2.4, projected CG): bounds lo = d_prev, hi = 1.
 * Each restart recomputes r = b - A x and the active set
 *   {x <= lo and r <= 0} U {x >= hi and r >= 0}   (ties count as active);
 * the solve has converged when the free-set residual satisfies
 * ||r_F||_2 <= tol ||b - A 1_D||_2.  Otherwise Jacobi-PCG runs on the free
 * set; after every update any free value outside [lo, hi] is projected back
 * and the solve restarts; a free-set CG that meets the tolerance also
 * restarts (which re-checks the active set).  *iters counts matvecs inside
 * the CG loops, *restarts the restarts. */
static int solve_at1(const or_mesh *m, const or_material *mt, const double *H,
                     const double *dprev, double *dout, const or_solve_opts *o,
                     int *iters, int *restarts, double *relres) {
  int64_t N = m->N;
  double *b = malloc(N * sizeof(double)), *dg = malloc(N * sizeof(double));
  double *x = malloc(N * sizeof(double)), *r = malloc(N * sizeof(double));
  double *z = malloc(N * sizeof(double)), *p = malloc(N * sizeof(double));
  double *q = malloc(N * sizeof(double)), *oneD = malloc(N * sizeof(double));
  uint8_t *nd = malloc(N), *fr = malloc(N);
  int st = OR_OK;
  for (int64_t i = 0; i < N; ++i) nd[i] = m->notch[i] ? 0 : 1;
  or_damage_rhs(m, mt, H, b, dg);
  for (int64_t i = 0; i < N; ++i) oneD[i] = nd[i] ? 0.0 : 1.0;
  or_damage_apply(m, mt, H, oneD, q);
  double bn2 = 0.0;
  for (int64_t i = 0; i < N; ++i)
    if (nd[i]) bn2 += (b[i] - q[i]) * (b[i] - q[i]);
  double bn = sqrt(bn2);
  for (int64_t i = 0; i < N; ++i) x[i] = nd[i] ? dprev[i] : 1.0;
  int k = 0, rs = 0;
  double rrF = 0.0;
  for (;;) {
    or_damage_apply(m, mt, H, x, q);
    for (int64_t i = 0; i < N; ++i) {
      r[i] = nd[i] ? b[i] - q[i] : 0.0;
      int act = nd[i] && ((x[i] <= dprev[i] && r[i] <= 0.0) || (x[i] >= 1.0 && r[i] >= 0.0));
      fr[i] = nd[i] && !act;
    }
    rrF = dot_free(m, fr, r, r);
    if (sqrt(rrF) <= o->tol * bn) break;
    if (rs >= o->max_restarts || k >= o->max_it) { st = OR_ERR_NOT_CONVERGED; break; }
    ++rs;
    for (int64_t i = 0; i < N; ++i) { z[i] = fr[i] ? r[i] / dg[i] : 0.0; p[i] = z[i]; }
    double rho = dot_free(m, fr, r, z);
    for (;;) {
      if (k >= o->max_it) break;
      or_damage_apply(m, mt, H, p, q);
      for (int64_t i = 0; i < N; ++i) if (!fr[i]) q[i] = 0.0;
      double pq = dot_free(m, fr, p, q);
      if (pq == 0.0) break;
      double alpha = rho / pq;
      int projected = 0;
      for (int64_t i = 0; i < N; ++i)
        if (fr[i]) {
          x[i] += alpha * p[i];
          r[i] -= alpha * q[i];
          if (x[i] < dprev[i]) { x[i] = dprev[i]; projected = 1; }
          if (x[i] > 1.0) { x[i] = 1.0; projected = 1; }
        }
      ++k;
      if (projected) break;
      double rr = dot_free(m, fr, r, r);
      if (sqrt(rr) <= o->tol * bn) break;
      for (int64_t i = 0; i < N; ++i) z[i] = fr[i] ? r[i] / dg[i] : 0.0;
      double rho_new = dot_free(m, fr, r, z);
      double beta = rho_new / rho;
      rho = rho_new;
      for (int64_t i = 0; i < N; ++i) p[i] = fr[i] ? z[i] + beta * p[i] : 0.0;
    }
  }
  *iters = k;
  *restarts = rs;
  *relres = bn > 0.0 ? sqrt(rrF) / bn : 0.0;
  for (int64_t i = 0; i < N; ++i) dout[i] = nd[i] ? x[i] : 1.0;
  free(b); free(dg); free(x); free(r); free(z); free(p); free(q); free(oneD);
  free(nd); free(fr);
  return st;
}

/* Public damage solve: model chosen from the material (Sec. 2.4 switches
 * AT2 -> post-clamp, AT1 -> projected CG).  info[0] = iterations,
 * info[1] = natural AT2 stop count or AT1 restarts. */
int or_damage_solve(const or_mesh *m, const or_material *mt, const double *H,
                    const double *dprev, double *dout, double tol, int max_it,
                    int max_restarts, int forced, int32_t *info, double *relres,
                    double *x_out) {
  or_solve_opts o = {tol, max_it, max_restarts};
  int it = 0, aux = 0, st;
  if (mt->model == OR_AT1)
    st = solve_at1(m, mt, H, dprev, dout, &o, &it, &aux, relres);
  else
    st = solve_at2(m, mt, H, dprev, dout, &o, forced, &it, &aux, relres, x_out);
  info[0] = it;
  info[1] = aux;
  return st;
}

/* ------------------------------------------------------------- energies */

/* out[0] = E_el = sum A_e psi(eps_e, dbar_e); out[1] = E_kin = 1/2 sum m v^2;
 * out[2] = E_frac = Gc * sum_e int gamma(d) over the element (AT2:
 * d^T M^e d / (2 l0) + l0/2 A_e |grad d|^2; AT1: 3/8 (A_e/3 sum d / l0 +
 * l0 A_e |grad d|^2)).  All per unit thickness (Sec. 3.1). */
void or_energies(const or_mesh *m, const or_material *mt, const double *mass,
                 const double *u, const double *v, const double *d, double *out) {
  double Eel = 0.0, Ekin = 0.0, Efr = 0.0;
  for (int64_t e = 0; e < m->Ne; ++e) {
    double eps[3], sig[3], sp[3], pp, pm, psi;
    elem_strain(m, e, u, eps);
    or_constitutive(mt, eps, elem_dbar(m, e, d), sig, sp, &pp, &pm, &psi);
    double A = m->area[e];
    Eel += A * psi;
    const double *g = m->grad + 6 * e;
    double gx = 0.0, gy = 0.0, de[3];
    for (int a = 0; a < 3; ++a) {
      de[a] = d[m->t[3 * e + a]];
      gx += g[2 * a] * de[a];
      gy += g[2 * a + 1] * de[a];
    }
    double grad2 = gx * gx + gy * gy;
    const double gc = elem_gc(m, mt, e);
    if (mt->model == OR_AT1) {
      Efr += gc * 0.375 * (A / 3.0 * (de[0] + de[1] + de[2]) / mt->l0 + mt->l0 * A * grad2);
    } else {
      double dMd = 0.0;
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) dMd += de[a] * de[b] * A * (a == b ? 2.0 : 1.0) / 12.0;
      Efr += gc * (dMd / (2.0 * mt->l0) + 0.5 * mt->l0 * A * grad2);
    }
  }
  for (int64_t i = 0; i < m->N; ++i)
    Ekin += 0.5 * mass[i] * (v[2 * i] * v[2 * i] + v[2 * i + 1] * v[2 * i + 1]);
  out[0] = Eel; out[1] = Ekin; out[2] = Efr;
}

/* --------------------------------------------- subcycling limit (check) */

/* Pre-simulation check of the damage subcycling factor (Sec. 2.4,
 * sec:subcycling): the damage front moves at most at about 0.6 c_R while
 * the explicit step is set by the dilatational speed c_p, so
 * N_max = floor(c_p / (0.6 c_R)).  c_p = sqrt((lambda + 2 mu) / rho) with
 * the plane model's lambda (the speed of the CFL step), c_s = sqrt(mu / rho),
 * c_R = xi c_s with xi in (0, 1) the root of the Rayleigh equation
 * (2 - xi^2)^2 = 4 sqrt(1 - k^2 xi^2) sqrt(1 - xi^2), k = c_s / c_p, found by
 * bisection (xi = 0 is a trivial root; the left side minus the right side
 * is negative just above 0 and positive at 1). */
void or_subcycling_limit(const or_material *mt, double *ratio, int32_t *nmax) {
  or_lame L = lame_of(mt);
  const double cp = sqrt((L.lam + 2.0 * L.mu) / mt->rho), cs = sqrt(L.mu / mt->rho);
  const double k = cs / cp;
  double lo = 1e-6, hi = 1.0;
  for (int it = 0; it < 200; ++it) {
    const double xi = 0.5 * (lo + hi), x2 = xi * xi;
    const double f = (2.0 - x2) * (2.0 - x2) - 4.0 * sqrt(1.0 - k * k * x2) * sqrt(1.0 - x2);
    if (f < 0.0) lo = xi; else hi = xi;
  }
  const double cR = 0.5 * (lo + hi) * cs;
  *ratio = cp / (0.6 * cR);
  *nmax = (int32_t)floor(*ratio);
}

/* ---------------------------------------------------------- time stepping */

typedef struct {
  double dt, t_ramp, tol;
  int32_t max_it, max_restarts;
  int32_t damage_on;     /* 0: skip the damage solve (d frozen) */
  int32_t energy_every;  /* 0: no energies */
  int32_t n_sub;         /* damage subcycling (Sec. 2.4, sec:subcycling):
                            the damage problem is solved only after steps
                            n with (n + 1) % n_sub == 0; 0 or 1: every step */
} or_run_opts;

/* One staggered step n -> n+1 (Sec. 2.2): predictor (vv_u), internal force
 * at u_{n+1} with d_n, history update, acceleration (vv_a), corrector
 * (vv_v), then the damage solve with H_{n+1}.  W_ext (nullable) accumulates
 * the trapezoid-rule external work.  x_out (nullable) receives the AT2
 * unclamped damage solution. */
static int step_once(const or_mesh *m, const or_material *mt, const double *minv,
                     const or_run_opts *o, int64_t n, double *u, double *v,
                     double *a, double *d, double *H, double *W, int forced,
                     int32_t *info, double *relres, double *f, double *psip,
                     double *dnew, double *x_out) {
  int64_t N = m->N;
  double S0 = or_ramp(n * o->dt, o->t_ramp), S1 = or_ramp((n + 1) * o->dt, o->t_ramp);
  for (int64_t i = 0; i < 2 * N; ++i) {
    double du = o->dt * v[i] + 0.5 * o->dt * o->dt * a[i];
    if (W) *W += 0.5 * (S0 + S1) * m->fext[i] * du;
    u[i] += du;
  }
  or_internal_force(m, mt, u, d, f, psip);
  for (int64_t e = 0; e < m->Ne; ++e)
    if (psip[e] > H[e]) H[e] = psip[e];
  for (int64_t i = 0; i < 2 * N; ++i) {
    double anew = minv[i / 2] * (S1 * m->fext[i] - f[i]);
    v[i] += 0.5 * o->dt * (a[i] + anew);
    a[i] = anew;
  }
  int st = OR_OK;
  info[0] = info[1] = 0;
  *relres = 0.0;
  /* subcycling: H above is still updated every step; d stays d_n between
     the solves */
  const int solve_now = o->n_sub <= 1 || (n + 1) % o->n_sub == 0;
  if (o->damage_on && solve_now) {
    st = or_damage_solve(m, mt, H, d, dnew, o->tol, o->max_it, o->max_restarts,
                         forced, info, relres, x_out);
    memcpy(d, dnew, N * sizeof(double));
  }
  return st;
}

/* Runs nsteps staggered steps in place on (u, v, a, d, H).
 * iters_log (nsteps x 2, nullable): info per step; relres_log (nullable);
 * energy_log (nsteps x 4, nullable): E_el, E_kin, E_frac, W_ext after each
 * step where (n+1) % energy_every == 0 (other rows untouched).
 * forced (nullable): per-step forced AT2 iteration counts.
 * Returns the worst status. */
int or_run(const or_mesh *m, const or_material *mt, const or_run_opts *o,
           int64_t n0, int64_t nsteps, double *u, double *v, double *a,
           double *d, double *H, int32_t *iters_log, double *relres_log,
           double *energy_log, const int32_t *forced, double *W_inout) {
  int64_t N = m->N;
  double *mass = malloc(N * sizeof(double)), *minv = malloc(N * sizeof(double));
  double *f = malloc(2 * N * sizeof(double)), *psip = malloc(m->Ne * sizeof(double));
  double *dnew = malloc(N * sizeof(double));
  or_lumped_mass(m, mt->rho, mass);
  for (int64_t i = 0; i < N; ++i) minv[i] = 1.0 / mass[i];
  double W = W_inout ? *W_inout : 0.0;
  int worst = OR_OK;
  for (int64_t s = 0; s < nsteps; ++s) {
    int32_t info[2];
    double rel;
    int st = step_once(m, mt, minv, o, n0 + s, u, v, a, d, H, &W,
                       forced ? forced[s] : -1, info, &rel, f, psip, dnew, NULL);
    if (st > worst) worst = st;
    if (iters_log) { iters_log[2 * s] = info[0]; iters_log[2 * s + 1] = info[1]; }
    if (relres_log) relres_log[s] = rel;
    if (energy_log && o->energy_every > 0 && (s + 1) % o->energy_every == 0) {
      or_energies(m, mt, mass, u, v, d, energy_log + 4 * s);
      energy_log[4 * s + 3] = W;
    }
  }
  if (W_inout) *W_inout = W;
  free(mass); free(minv); free(f); free(psip); free(dnew);
  return worst;
}

/* ------------------------------------------------------------- adjoint */

/* Jacobi-PCG for A lam = g on the free (non-notch) nodes to a tight
 * tolerance; the adjoint solve of Eq. (implicit_adjoint_linear_system)
 * (A is symmetric, so A^T = A). */
static void adjoint_solve(const or_mesh *m, const or_material *mt, const double *H,
                          const double *g, double *lam) {
  int64_t N = m->N;
  double *b = malloc(N * sizeof(double)), *dg = malloc(N * sizeof(double));
  double *r = malloc(N * sizeof(double)), *z = malloc(N * sizeof(double));
  double *p = malloc(N * sizeof(double)), *q = malloc(N * sizeof(double));
  uint8_t *fr = malloc(N);
  for (int64_t i = 0; i < N; ++i) fr[i] = m->notch[i] ? 0 : 1;
  or_damage_rhs(m, mt, H, b, dg);
  for (int64_t i = 0; i < N; ++i) { lam[i] = 0.0; r[i] = fr[i] ? g[i] : 0.0; }
  double gn = sqrt(dot_free(m, fr, r, r));
  if (gn > 0.0) {
    for (int64_t i = 0; i < N; ++i) { z[i] = fr[i] ? r[i] / dg[i] : 0.0; p[i] = z[i]; }
    double rho = dot_free(m, fr, r, z);
    for (int k = 0; k < 100000; ++k) {
      or_damage_apply(m, mt, H, p, q);
      for (int64_t i = 0; i < N; ++i) if (!fr[i]) q[i] = 0.0;
      double pq = dot_free(m, fr, p, q);
      if (pq == 0.0) break;
      double alpha = rho / pq;
      for (int64_t i = 0; i < N; ++i)
        if (fr[i]) { lam[i] += alpha * p[i]; r[i] -= alpha * q[i]; }
      if (sqrt(dot_free(m, fr, r, r)) <= 1e-15 * gn) break;
      for (int64_t i = 0; i < N; ++i) z[i] = fr[i] ? r[i] / dg[i] : 0.0;
      double rho_new = dot_free(m, fr, r, z);
      double beta = rho_new / rho;
      rho = rho_new;
      for (int64_t i = 0; i < N; ++i) p[i] = fr[i] ? z[i] + beta * p[i] : 0.0;
    }
  }
  free(b); free(dg); free(r); free(z); free(p); free(q); free(fr);
}

/* Parameter and history terms of the implicit damage adjoint (AT2):
 *   dL/dGc_e += -lam_e^T (l0 K^e + M^e / l0) xt_e (Eq. implicit_gc_l0_element_term,
 *               per element; their sum is dL/dGc for a uniform Gc)
 *   Hbar_e  += (2 A_e / 3) sum_a lam_a - 2 lam_e^T M^e xt_e
 * with xt = the unclamped solution on free nodes and 1 on the notch.
 * gce_bar (Ne, nullable) accumulates the per-element terms. */
void or_damage_adjoint_terms(const or_mesh *m, const or_material *mt,
                             const double *lam, const double *xt,
                             double *gc_bar, double *Hbar, double *gce_bar) {
  double acc = 0.0;
  for (int64_t e = 0; e < m->Ne; ++e) {
    const double *g = m->grad + 6 * e;
    double A = m->area[e];
    double sK = 0.0, sM = 0.0, slam = 0.0;
    for (int a = 0; a < 3; ++a) {
      double la = lam[m->t[3 * e + a]];
      slam += la;
      for (int b = 0; b < 3; ++b) {
        double xb = xt[m->t[3 * e + b]];
        double Kab = A * (g[2 * a] * g[2 * b] + g[2 * a + 1] * g[2 * b + 1]);
        double Mab = A * (a == b ? 2.0 : 1.0) / 12.0;
        sK += la * Kab * xb;
        sM += la * Mab * xb;
      }
    }
    const double te = -(mt->l0 * sK + sM / mt->l0);
    acc += te;
    if (gce_bar) gce_bar[e] += te;
    Hbar[e] += 2.0 * A / 3.0 * slam - 2.0 * sM;
  }
  *gc_bar += acc;
}

/* Reverse of the element force (the symmetric Hessian of sum A_e psi):
 * for each element, de = sym grad(fbar_e), and
 *   ubar_a += A_e Dsigma[de] . grad phi_a + psibar_e sigma+ . grad phi_a
 *   dbar_a += (1/3) g'(dbar_e) A_e (de : sigma+)
 * accumulated in element order.  u is u_{n+1}, d is d_n. */
void or_elem_adjoint(const or_mesh *m, const or_material *mt, const double *u,
                     const double *d, const double *fbar, const double *psibar,
                     double *ubar, double *dbar) {
  for (int64_t e = 0; e < m->Ne; ++e) {
    double eps[3], de[3], sp[3], sm[3], pp, pm, ds[3];
    elem_strain(m, e, u, eps);
    elem_strain(m, e, fbar, de);
    split_point(mt, eps, sp, sm, &pp, &pm);
    double db = elem_dbar(m, e, d);
    or_constitutive_tangent(mt, eps, db, de, ds);
    double A = m->area[e];
    double pb = psibar ? psibar[e] : 0.0;
    double gprime = -2.0 * (1.0 - db);
    double dterm = gprime * A * (de[0] * sp[0] + de[1] * sp[1] + 2.0 * de[2] * sp[2]) / 3.0;
    const double *g = m->grad + 6 * e;
    for (int a = 0; a < 3; ++a) {
      int32_t n = m->t[3 * e + a];
      double sx = A * ds[0] + pb * sp[0], sy = A * ds[1] + pb * sp[1], sxy = A * ds[2] + pb * sp[2];
      ubar[2 * n] += sx * g[2 * a] + sxy * g[2 * a + 1];
      ubar[2 * n + 1] += sxy * g[2 * a] + sy * g[2 * a + 1];
      dbar[n] += dterm;
    }
  }
}

/* dL/dGc of L = (1/N) sum_i (d_T,i - dstar_i)^2 after nsteps AT2 steps from
 * the given initial state, by the discrete adjoint of the realised
 * trajectory (Sec. 4.2): every state is stored, the damage solve is treated
 * as exact (Eq. implicit_adjoint_linear_system), the history max passes its
 * gradient to psi+ only where psi+ > H_n, and the clamp passes it to the
 * solution only where d_n < x < 1 (to d_n where x <= d_n).
 * Returns the loss in *loss and the gradient in *dL_dGc; *status gets the
 * forward's worst status. */
int or_adjoint_gc(const or_mesh *m, const or_material *mt, const or_run_opts *o,
                  int64_t nsteps, const double *u0, const double *v0,
                  const double *a0, const double *d0, const double *H0,
                  const double *dstar, double *loss, double *dL_dGc,
                  double *dL_dGc_field) {
  int64_t N = m->N, Ne = m->Ne, T = nsteps;
  if (dL_dGc_field) memset(dL_dGc_field, 0, Ne * sizeof(double));
  double *U = malloc((T + 1) * 2 * N * sizeof(double));
  double *D = malloc((T + 1) * N * sizeof(double));
  double *HS = malloc((T + 1) * Ne * sizeof(double));
  double *X = malloc((T + 1) * N * sizeof(double));
  double *v = malloc(2 * N * sizeof(double)), *a = malloc(2 * N * sizeof(double));
  double *mass = malloc(N * sizeof(double)), *minv = malloc(N * sizeof(double));
  double *f = malloc(2 * N * sizeof(double)), *psip = malloc(Ne * sizeof(double));
  double *dnew = malloc(N * sizeof(double));
  or_lumped_mass(m, mt->rho, mass);
  for (int64_t i = 0; i < N; ++i) minv[i] = 1.0 / mass[i];
  memcpy(U, u0, 2 * N * sizeof(double));
  memcpy(v, v0, 2 * N * sizeof(double));
  memcpy(a, a0, 2 * N * sizeof(double));
  memcpy(D, d0, N * sizeof(double));
  memcpy(HS, H0, Ne * sizeof(double));
  int worst = OR_OK;
  for (int64_t n = 0; n < T; ++n) {
    double *u = U + (n + 1) * 2 * N, *d = D + (n + 1) * N, *H = HS + (n + 1) * Ne;
    memcpy(u, U + n * 2 * N, 2 * N * sizeof(double));
    memcpy(d, D + n * N, N * sizeof(double));
    memcpy(H, HS + n * Ne, Ne * sizeof(double));
    int32_t info[2];
    double rel;
    int st = step_once(m, mt, minv, o, n, u, v, a, d, H, NULL, -1, info, &rel,
                       f, psip, dnew, X + (n + 1) * N);
    if (st > worst) worst = st;
  }
  double L = 0.0;
  for (int64_t i = 0; i < N; ++i) {
    double r = D[T * N + i] - dstar[i];
    L += r * r;
  }
  *loss = L / N;

  double *ub = calloc(2 * N, sizeof(double)), *vb = calloc(2 * N, sizeof(double));
  double *ab = calloc(2 * N, sizeof(double)), *db = calloc(N, sizeof(double));
  double *Hb = calloc(Ne, sizeof(double));
  double *xbar = malloc(N * sizeof(double)), *lam = malloc(N * sizeof(double));
  double *xt = malloc(N * sizeof(double)), *fbar = malloc(2 * N * sizeof(double));
  double *pbar = malloc(Ne * sizeof(double)), *ubn = malloc(2 * N * sizeof(double));
  double *dbn = malloc(N * sizeof(double));
  for (int64_t i = 0; i < N; ++i) db[i] = 2.0 * (D[T * N + i] - dstar[i]) / N;
  double gc = 0.0;
  for (int64_t n = T - 1; n >= 0; --n) {
    const double *u1 = U + (n + 1) * 2 * N, *dn = D + n * N;
    const double *Hn = HS + n * Ne, *H1 = HS + (n + 1) * Ne, *x = X + (n + 1) * N;
    /* damage: clamp masks, adjoint solve, parameter and history terms */
    for (int64_t i = 0; i < N; ++i) {
      dbn[i] = 0.0;
      xbar[i] = 0.0;
      if (m->notch[i]) continue;
      if (x[i] > dn[i] && x[i] < 1.0) xbar[i] = db[i];
      else if (x[i] <= dn[i]) dbn[i] = db[i];
    }
    adjoint_solve(m, mt, H1, xbar, lam);
    for (int64_t i = 0; i < N; ++i) xt[i] = m->notch[i] ? 1.0 : x[i];
    or_damage_adjoint_terms(m, mt, lam, xt, &gc, Hb, dL_dGc_field);
    /* corrector and acceleration: fbar = -minv (abar + dt/2 vbar) */
    for (int64_t i = 0; i < 2 * N; ++i)
      fbar[i] = -minv[i / 2] * (ab[i] + 0.5 * o->dt * vb[i]);
    /* history max: psi+ > H_n passes Hbar to psi+, else to H_n */
    or_internal_force(m, mt, u1, dn, f, psip);
    for (int64_t e = 0; e < Ne; ++e) {
      if (psip[e] > Hn[e]) { pbar[e] = Hb[e]; Hb[e] = 0.0; }
      else pbar[e] = 0.0;
    }
    (void)H1;
    /* element force reverse */
    memcpy(ubn, ub, 2 * N * sizeof(double));
    or_elem_adjoint(m, mt, u1, dn, fbar, pbar, ubn, dbn);
    /* predictor reverse */
    for (int64_t i = 0; i < 2 * N; ++i) {
      double vbar_next = vb[i];
      ub[i] = ubn[i];
      vb[i] = vbar_next + o->dt * ubn[i];
      ab[i] = 0.5 * o->dt * vbar_next + 0.5 * o->dt * o->dt * ubn[i];
    }
    memcpy(db, dbn, N * sizeof(double));
  }
  *dL_dGc = gc;
  free(U); free(D); free(HS); free(X); free(v); free(a); free(mass); free(minv);
  free(f); free(psip); free(dnew); free(ub); free(vb); free(ab); free(db); free(Hb);
  free(xbar); free(lam); free(xt); free(fbar); free(pbar); free(ubn); free(dbn);
  return worst;
}
