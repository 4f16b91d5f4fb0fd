// adjoint.cuh -- reverse (adjoint) kernels of the staggered step, sm_103a.
//
// Differentiates the realised discrete trajectory (Sec. 4) for dL/dGc:
//  * damage solve: implicit differentiation, Eqs.
//    (implicit_forward_linear_system) and (implicit_adjoint_linear_system):
//    one adjoint CG solve A(H_{n+1}) lam = g per step (A is symmetric), with
//    the parameter term of Eq. (implicit_gc_l0_element_term) and the history
//    term, both per element;
//  * active-set masking (Sec. 4.2): the clamp passes the gradient to the
//    solution where d_n < x < 1, to d_n where x <= d_n; the history max
//    passes it to psi+ only where psi+ > H_n (read off the stored H's);
//  * explicit mechanics: the reverse of the predictor and corrector (Eqs.
//    vv_u, vv_a, vv_v) and of the element force, whose Jacobian is the
//    symmetric tangent of the split energy (the Hessian of A_e psi), applied
//    node-centrically with the same incidence gather as the forward.
#pragma once
#include "kernels.cuh"

namespace pff {

template <typename R> struct AdjParams {
  typedef typename V<R>::T2 R2;
  Params<R> P;  // mesh, material, CG workspace (x = lambda), solve scalars
  // tape of the current segment: slot k holds u_{n+1}, x_{n+1}, d_{n+1},
  // H_{n+1} of step n = s0 + k; slot -1 is the segment's checkpoint (d, H).
  // The slot of the step being reversed is read from *kctr.
  const int *kctr;
  int *kdec;    // = kctr: decremented by the last block of the reverse step
  const R2 *tape_u;
  const R *tape_x, *tape_d;
  const double *tape_H;
  const R *snap_d;
  const double *snap_H;
  int32_t stride_n, stride_e;  // slot strides (elements of R2/R, doubles)
  const int64_t *x_base;       // nullable: tape_x holds the whole run, slot k of
                               // this segment at *x_base + k (damage-tape policy)
  R *Hcur;                     // H_{n+1} in the kernel precision (operator)
  int32_t h_tape;              // 1: k_adj_rhs reads H_{n+1} from the tape (no Hcur)
  // adjoint state (in: step n+1, out: step n)
  const R2 *ub_in, *vb_in, *ab_in;
  R2 *ub_out, *vb_out, *ab_out;
  R *db;             // dL/dd: in d_{n+1}, out d_n
  R *dbn;            // clamp share of dL/dd_n
  R *g;              // right-hand side of the adjoint solve
  const R *Hb_in;    // dL/dH_{n+1} from the later steps (before this step's damage terms)
  R *Hb_out;         // dL/dH_n
  R2 *fe;            // 3 Ne: the element shares of ubar per slot (reverse mechanics)
  R *fd;             // Ne: the element shares of dbar
  double *gc;        // running dL/dGc
  double *gce;       // running dL/dGc_e per element (nullable)
  int *astat;        // worst status of the adjoint solves (atomicMax)
};

template <typename R> struct Slot {
  const typename V<R>::T2 *u1;
  const R *x1, *d0;
  const double *H0, *H1;
};

template <typename R>
__device__ __forceinline__ Slot<R> slot(const AdjParams<R> &A) {
  const int k = *A.kctr;
  Slot<R> s;
  s.u1 = A.tape_u + (size_t)k * A.stride_n;
  s.x1 = A.tape_x + (size_t)((A.x_base ? *A.x_base : 0) + k) * A.stride_n;
  s.H1 = A.tape_H + (size_t)k * A.stride_e;
  s.d0 = k > 0 ? A.tape_d + (size_t)(k - 1) * A.stride_n : A.snap_d;
  s.H0 = k > 0 ? A.tape_H + (size_t)(k - 1) * A.stride_e : A.snap_H;
  return s;
}

// H_{n+1} of the current slot in the kernel precision (the adjoint
// operator's history, for the solves that read it from P.Hr).
template <typename R>
__global__ void __launch_bounds__(256) k_adj_load(AdjParams<R> A) {
  const Slot<R> S = slot(A);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < A.P.Ne; e += gridDim.x * blockDim.x)
    A.Hcur[e] = (R)S.H1[e];
}

// Splits at one point: sigma+, sigma- and psi+ (same formulas as stress()).
template <typename R>
__device__ __forceinline__ void split_parts(const Params<R> &P, R exx, R eyy, R exy, R (&sp)[3], R (&sm)[3]) {
  R sxx, syy, sxy, psip;
  stress(P, exx, eyy, exy, R(1), sxx, syy, sxy, psip);  // sigma+ + sigma-
  R fxx, fyy, fxy, dummy;
  stress(P, exx, eyy, exy, R(0), fxx, fyy, fxy, dummy);  // sigma-
  sm[0] = fxx;
  sm[1] = fyy;
  sm[2] = fxy;
  sp[0] = sxx - fxx;
  sp[1] = syy - fyy;
  sp[2] = sxy - fxy;
}

// Tangent action of the split, dsigma+[de] and dsigma-[de] (the Hessian of
// psi+/psi- applied to de).  Spectral: with n = D / |D| the unit deviator,
// d eps+ = H1 (P1:de) P1 + H2 (P2:de) P2 + theta/2 (de - n de n), theta =
// (<e1>+ - <e2>+)/(e1 - e2); kinks use <x>+'(0) = 0 and a double principal
// strain the limit H(e1).
template <typename R>
__device__ __forceinline__ void split_tangent(const Params<R> &P, R exx, R eyy, R exy, const R (&de)[3],
                                              R (&dsp)[3], R (&dsm)[3]) {
  const R tr = exx + eyy, dtr = de[0] + de[1];
  const R Htr = tr > R(0) ? R(1) : R(0);
  if (P.split == kSpectral) {
    const R half = R(0.5) * (exx - eyy);
    const R rad = sqrt(half * half + exy * exy);
    const R e1 = R(0.5) * tr + rad, e2 = R(0.5) * tr - rad;
    const R H1 = e1 > R(0) ? R(1) : R(0), H2 = e2 > R(0) ? R(1) : R(0);
    R dxx, dyy, dxy;
    if (rad > R(0)) {
      const R a = half / rad, b = exy / rad;
      const R nd = a * (de[0] - de[1]) + R(2) * b * de[2];    // n : de
      const R p1d = R(0.5) * (dtr + nd), p2d = R(0.5) * (dtr - nd);
      const R theta = (rpos(e1) - rpos(e2)) / (R(2) * rad);
      // n de n
      const R ndn_xx = a * a * de[0] + R(2) * a * b * de[2] + b * b * de[1];
      const R ndn_yy = b * b * de[0] - R(2) * a * b * de[2] + a * a * de[1];
      const R ndn_xy = a * b * (de[0] - de[1]) + (b * b - a * a) * de[2];
      // P1 = (I + n)/2, P2 = (I - n)/2
      dxx = H1 * p1d * R(0.5) * (R(1) + a) + H2 * p2d * R(0.5) * (R(1) - a) + R(0.5) * theta * (de[0] - ndn_xx);
      dyy = H1 * p1d * R(0.5) * (R(1) - a) + H2 * p2d * R(0.5) * (R(1) + a) + R(0.5) * theta * (de[1] - ndn_yy);
      dxy = H1 * p1d * R(0.5) * b - H2 * p2d * R(0.5) * b + R(0.5) * theta * (de[2] - ndn_xy);
    } else {
      dxx = H1 * de[0];
      dyy = H1 * de[1];
      dxy = H1 * de[2];
    }
    const R mu2 = R(2) * P.mu;
    dsp[0] = P.lam * Htr * dtr + mu2 * dxx;
    dsp[1] = P.lam * Htr * dtr + mu2 * dyy;
    dsp[2] = mu2 * dxy;
    dsm[0] = P.lam * (R(1) - Htr) * dtr + mu2 * (de[0] - dxx);
    dsm[1] = P.lam * (R(1) - Htr) * dtr + mu2 * (de[1] - dyy);
    dsm[2] = mu2 * (de[2] - dxy);
  } else if (P.split == kAmor && P.cz == R(0)) {
    const R mu2 = R(2) * P.mu, t3 = dtr * (R(1) / R(3));
    dsp[0] = P.K * Htr * dtr + mu2 * (de[0] - t3);
    dsp[1] = P.K * Htr * dtr + mu2 * (de[1] - t3);
    dsp[2] = mu2 * de[2];
    dsm[0] = P.K * (R(1) - Htr) * dtr;
    dsm[1] = P.K * (R(1) - Htr) * dtr;
    dsm[2] = R(0);
  } else if (P.split == kAmor) {
    // plane stress (see stress()): tr3 = f tr, e_zz = -cz tr
    const R f = R(1) - P.cz, mu2 = R(2) * P.mu;
    const R H3 = f * tr > R(0) ? R(1) : R(0);
    const R lin = (P.cz * P.cz - f * f * (R(1) / R(3))) * dtr;
    dsp[0] = P.K * H3 * f * f * dtr + mu2 * (de[0] + lin);
    dsp[1] = P.K * H3 * f * f * dtr + mu2 * (de[1] + lin);
    dsp[2] = mu2 * de[2];
    dsm[0] = P.K * (R(1) - H3) * f * f * dtr;
    dsm[1] = P.K * (R(1) - H3) * f * f * dtr;
    dsm[2] = R(0);
  } else {
    const R mu2 = R(2) * P.mu;
    dsp[0] = P.lam * dtr + mu2 * de[0];
    dsp[1] = P.lam * dtr + mu2 * de[1];
    dsp[2] = mu2 * de[2];
    dsm[0] = dsm[1] = dsm[2] = R(0);
  }
}

// One incidence entry (slot k of node i) of the adjoint solve's set-up: its
// share of the Jacobi diagonal and of A lam0 (the operator at H_{n+1},
// Eqs. damage_pde_at2 / matrix_free_fe_operator), writing the solve's FP32
// entry record.
template <typename R>
__device__ __forceinline__ void adj_rhs_entry(const AdjParams<R> &A, const Slot<R> &S, int en, int k, int i,
                                              R &dgc, R &axc, typename Params<R>::R2 *cf, uint32_t fm) {
  typedef typename Params<R>::R4 R4;
  const Params<R> &P = A.P;
  const int e = en >> 2, a = en & 3;
  int4 t;
  R Ar;
  R4 G;
  load_elem(P, e, t, Ar, G);
  const R sg = gc_scale(P, e);
  const R c = P.cbase * sg + R(2) * (A.h_tape ? (R)S.H1[e] : P.Hr[e]);
  const R kA = (P.kappa * sg) * Ar, mA = c * Ar * (R(1) / R(12));
  R gx, gy;
  slot_grad<R>(G, a, gx, gy);
  dgc = kA * (gx * gx + gy * gy) + R(2) * mA;
  if (cf)
    *cf = erec_coef<R>(G, a, kA, mA);
  else if (has_erec(P))
    put_erec(P, k, i, G, a, kA, mA, fm);
  const R l0 = (P.flags[t.x] & kNotch) ? R(0) : P.x[t.x];
  const R l1 = (P.flags[t.y] & kNotch) ? R(0) : P.x[t.y];
  const R l2 = (P.flags[t.z] & kNotch) ? R(0) : P.x[t.z];
  axc = elem_row<R>(G, a, kA, mA, l0, l1, l2);
}

// Adjoint solve set-up (same operator as the forward damage solve at
// H_{n+1}): per node the right-hand side and the clamp share of dL/dd_n,
//   g = dL/dd_{n+1} where d_n < x_{n+1} < 1 (free nodes), else 0;
//   dbn = dL/dd_{n+1} where x_{n+1} <= d_n (free nodes), else 0;
// warm start lam0 = previous lambda (in P.x), r = g - A lam0, Jacobi
// diagonal, z, p = 0; reductions |g|^2, |r|^2, r.z.
template <typename R>
__global__ void __launch_bounds__(256) k_adj_rhs(AdjParams<R> A) {
  typedef typename Params<R>::R4 R4;
  typedef Acc<R> AC;
  const Params<R> &P = A.P;
  const Slot<R> S = slot(A);
  typename AC::T vals[3] = {AC::zero(), AC::zero(), AC::zero()};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.N; i += gridDim.x * blockDim.x) {
    R gi = R(0), bi = R(0);
    if (!(P.flags[i] & kNotch)) {
      const R x = S.x1[i], lo = S.d0[i], db = A.db[i];
      if (x > lo && x < R(1)) gi = db;
      else if (x <= lo) bi = db;
    }
    A.g[i] = gi;
    A.dbn[i] = bi;
    if (P.flags[i] & kNotch) {
      P.x[i] = R(0);
      P.r[i] = R(0);
      typename Params<R>::R2 w;
      w.x = R(0);
      w.y = R(0);
      P.pz[i] = w;
      P.dinv[i] = R(0);
      continue;
    }
    R dg = 0, ax = 0;
    const bool merge = nb_merging(P);
    NbAcc<R> nacc;
    nacc.zero();
    if (merge) nacc.load_map(P, i);
    const uint32_t fm = fan_word(P, i);
    // two incidence entries in flight, summed in slot order
    for (int k = 0; k < P.D; k += 2) {
      int en[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) en[u] = k + u < P.D ? __ldg(&P.ell[(size_t)(k + u) * P.N + i]) : -1;
      R cd[2], ca[2];
      typename Params<R>::R2 cf[2];
#pragma unroll
      for (int u = 0; u < 2; ++u)
        if (en[u] >= 0) adj_rhs_entry(A, S, en[u], k + u, i, cd[u], ca[u], merge ? &cf[u] : nullptr, fm);
#pragma unroll
      for (int u = 0; u < 2; ++u)
        if (en[u] >= 0) {
          dg = radd(dg, cd[u]);
          ax = radd(ax, ca[u]);
          if (merge) nacc.add(k + u, cf[u]);
        }
    }
    const R ri = gi - ax, di = R(1) / dg, zi = ri * di;
    if (P.diag) P.diag[i] = dg;
    if (merge) nacc.store(P, i);
    P.r[i] = ri;
    P.dinv[i] = di;
    typename Params<R>::R2 w;
    w.x = R(0);
    w.y = zi;
    P.pz[i] = w;
    const R sr = P.rscale * ri, sg = P.rscale * gi;
    vals[0] = AC::add(vals[0], AC::prod(sg, sg));
    vals[1] = AC::add(vals[1], AC::prod(sr, sr));
    vals[2] = AC::add(vals[2], AC::prod(sr, zi));
  }
  __shared__ double tot[3];
  if (reduce_last<R, 3>(vals, P.part, P.ticket, tot) && threadIdx.x == 0) {
    SolveScalars &S = *P.sc;
    S.bn = sqrt(tot[0]);
    S.rr = tot[1];
    S.rho = tot[2];
    S.beta = 0.0;
    S.alpha = 0.0;
    S.beta_f = 0.f;
    S.alpha_f = 0.f;
    S.iters = 0;
    S.restarts = 0;
    S.status = kStOk;
    S.projected = 0;
    S.bar = 0u;
    S.abort = 0;
    const bool done = S.bn == 0.0 || sqrt(S.rr) <= P.tol * S.bn;
    S.done = done ? 1 : 0;
    if (P.use_cond) cudaGraphSetConditional(P.cond_inner, done ? 0u : 1u);
  }
}

// Parameter and history terms of the damage adjoint for element e (AT2;
// Eq. implicit_gc_l0_element_term and the H-derivative of A and b):
//   gterm = lam_e^T (l0 K^e + M^e / l0) xt_e  (dL/dGc -= gterm; per element
//   the derivative with respect to Gc_e of a toughness field),
//   Hbar_e += (2 A_e / 3) sum_a lam_a - 2 lam_e^T M^e xt_e,
// with xt = x_{n+1} on free nodes and 1 on the notch, M^e = A_e (1+delta)/12;
// lam = 0 when the solve's right-hand side was 0 (the CG stopped at once and
// left the warm start).  Returns Hbar_e with this step's terms.
template <typename R>
__device__ __forceinline__ R adj_dmg_terms(const AdjParams<R> &A, const Slot<R> &S, const int4 &t, R Ar,
                                           const typename Params<R>::R4 &G, bool zero_lam, R hb_in, R &gterm) {
  const Params<R> &P = A.P;
  const bool n0 = P.flags[t.x] & kNotch, n1 = P.flags[t.y] & kNotch, n2 = P.flags[t.z] & kNotch;
  const R la0 = (n0 || zero_lam) ? R(0) : P.x[t.x];
  const R la1 = (n1 || zero_lam) ? R(0) : P.x[t.y];
  const R la2 = (n2 || zero_lam) ? R(0) : P.x[t.z];
  const R x0 = n0 ? R(1) : S.x1[t.x], x1 = n1 ? R(1) : S.x1[t.y], x2 = n2 ? R(1) : S.x1[t.z];
  // lam^T K^e xt with K^e = A grad(phi) grad(phi)^T: A (grad lam).(grad xt)
  const R glx = G.x * (la0 - la2) + G.z * (la1 - la2), gly = G.y * (la0 - la2) + G.w * (la1 - la2);
  const R gxx = G.x * (x0 - x2) + G.z * (x1 - x2), gxy = G.y * (x0 - x2) + G.w * (x1 - x2);
  const R lKx = Ar * (glx * gxx + gly * gxy);
  // lam^T M^e xt = A/12 (sum lam_a x_a + sum lam . sum x)
  const R sl = la0 + la1 + la2, sx = x0 + x1 + x2;
  const R lMx = Ar * (R(1) / R(12)) * (la0 * x0 + la1 * x1 + la2 * x2 + sl * sx);
  gterm = (R)P.l0 * lKx + (R(1) / (R)P.l0) * lMx;
  return hb_in + R(2) * Ar * (R(1) / R(3)) * sl - R(2) * lMx;
}

// fbar at node j: -(1/m_j) (abar_j + dt/2 vbar_j).
template <typename R>
__device__ __forceinline__ typename Params<R>::R2 fbar_at(const AdjParams<R> &A, int j, R hdt) {
  const typename Params<R>::R2 ab = A.ab_in[j], vb = A.vb_in[j];
  const R mi = A.P.minv[j];
  typename Params<R>::R2 f;
  f.x = -mi * (ab.x + hdt * vb.x);
  f.y = -mi * (ab.y + hdt * vb.y);
  return f;
}

// Reverse of the mechanics of step n -> n+1, element pass (one thread per
// element): with de_e = sym grad(fbar) on element e, dsigma = g dsigma+ +
// dsigma-, and psibar_e = Hbar_e where H_{n+1,e} > H_{n,e} (the max picked
// psi+), the element's share of ubar at its slot a,
//   A_e dsigma[de_e] . grad(phi_a) + psibar_e sigma+_e . grad(phi_a),
// goes to fe[3e + a], and its share of dbar at each of its nodes,
//   g'(dbar_e) A_e (de_e : sigma+_e) / 3, to fd[e].  Hbar_e comes with the
// step's damage terms (adj_dmg_terms); Hbar_n and the element's Gc term (to
// dL/dGc and the per-element gradient) are written here.  The last block
// adds the summed Gc terms and records the solve's status and iterations.
template <typename R>
__global__ void __launch_bounds__(256) k_adj_mech_elem(AdjParams<R> A) {
  typedef typename Params<R>::R2 R2;
  typedef typename Params<R>::R4 R4;
  typedef Acc<R> AC;
  const Params<R> &P = A.P;
  const Slot<R> S = slot(A);
  const R hdt = R(0.5) * (R)P.dt;
  const bool zero_lam = P.sc->bn == 0.0;
  typename AC::T vals[1] = {AC::zero()};
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < P.Ne; e += gridDim.x * blockDim.x) {
    int4 t;
    R Ar;
    R4 G;
    load_elem(P, e, t, Ar, G);
    // strain of u_{n+1}
    const R2 u0 = S.u1[t.x], u1 = S.u1[t.y], u2 = S.u1[t.z];
    R ax0 = u0.x - u2.x, ax1 = u1.x - u2.x, ay0 = u0.y - u2.y, ay1 = u1.y - u2.y;
    const R exx = G.x * ax0 + G.z * ax1, eyy = G.y * ay0 + G.w * ay1;
    const R exy = R(0.5) * (G.y * ax0 + G.w * ax1 + G.x * ay0 + G.z * ay1);
    // strain of fbar
    const R2 f0 = fbar_at(A, t.x, hdt), f1 = fbar_at(A, t.y, hdt), f2 = fbar_at(A, t.z, hdt);
    ax0 = f0.x - f2.x; ax1 = f1.x - f2.x; ay0 = f0.y - f2.y; ay1 = f1.y - f2.y;
    R de[3];
    de[0] = G.x * ax0 + G.z * ax1;
    de[1] = G.y * ay0 + G.w * ay1;
    de[2] = R(0.5) * (G.y * ax0 + G.w * ax1 + G.x * ay0 + G.z * ay1);
    const R db = (S.d0[t.x] + S.d0[t.y] + S.d0[t.z]) * (R(1) / R(3));
    const R g = (R(1) - db) * (R(1) - db) + P.eta, gp = R(-2) * (R(1) - db);
    R sp[3], sm[3], dsp[3], dsm[3];
    split_parts(P, exx, eyy, exy, sp, sm);
    split_tangent(P, exx, eyy, exy, de, dsp, dsm);
    // the forward's max picked psi+ exactly where H grew (non-negative
    // doubles compare like their bit patterns)
    const bool picked = __double_as_longlong(S.H1[e]) > __double_as_longlong(S.H0[e]);
    R gterm;
    const R hb = adj_dmg_terms(A, S, t, Ar, G, zero_lam, A.Hb_in[e], gterm);
    const R pb = picked ? hb : R(0);
    const R sx = Ar * (g * dsp[0] + dsm[0]) + pb * sp[0];
    const R sy = Ar * (g * dsp[1] + dsm[1]) + pb * sp[1];
    const R sxy = Ar * (g * dsp[2] + dsm[2]) + pb * sp[2];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      R gx, gy;
      slot_grad<R>(G, a, gx, gy);
      R2 f;
      f.x = sx * gx + sxy * gy;
      f.y = sxy * gx + sy * gy;
      A.fe[(size_t)3 * e + a] = f;
    }
    A.fd[e] = gp * Ar * (de[0] * sp[0] + de[1] * sp[1] + R(2) * de[2] * sp[2]) * (R(1) / R(3));
    A.Hb_out[e] = picked ? R(0) : hb;
    vals[0] = AC::add(vals[0], AC::prod(R(-1), gterm));
    if (A.gce) A.gce[e] -= (double)gterm;
  }
  __shared__ double tot[1];
  if (reduce_last<R, 1>(vals, P.part, P.ticket, tot) && threadIdx.x == 0) {
    *A.gc += tot[0];
    if (A.astat) {
      if (P.sc->status) atomicMax(A.astat, P.sc->status);
      atomicAdd(A.astat + 1, P.sc->iters);  // adjoint CG iterations, summed
    }
  }
}

// Reverse of the mechanics, node pass: ubar' = ubar_{n+1} + the element
// shares at node i (incidence order, ascending element),
//   dbar_n = dbn + the element shares fd, vbar_n = vbar_{n+1} + dt ubar',
//   abar_n = dt/2 vbar_{n+1} + dt^2/2 ubar', ubar_n = ubar'.  The last block
// to finish moves the slot counter to the previous step (every block has
// read the slot by then).
template <typename R>
__global__ void __launch_bounds__(256) k_adj_mech_node(AdjParams<R> A) {
  typedef typename Params<R>::R2 R2;
  const Params<R> &P = A.P;
  const R dt = (R)P.dt, hdt = R(0.5) * dt;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.N; i += gridDim.x * blockDim.x) {
    R ux = 0, uy = 0, dsum = 0;
    // four incidence entries in flight, summed in slot order
    for (int k = 0; k < P.D; k += 4) {
      int en[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) en[u] = k + u < P.D ? __ldg(&P.ell[(size_t)(k + u) * P.N + i]) : -1;
      R2 f[4];
      R fdv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (en[u] >= 0) {
          f[u] = A.fe[(size_t)3 * (en[u] >> 2) + (en[u] & 3)];
          fdv[u] = A.fd[en[u] >> 2];
        }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (en[u] >= 0) {
          ux = radd(ux, f[u].x);
          uy = radd(uy, f[u].y);
          dsum = radd(dsum, fdv[u]);
        }
    }
    const R2 ubi = A.ub_in[i], vbi = A.vb_in[i];
    R2 up, vo, ao;
    up.x = ubi.x + ux;
    up.y = ubi.y + uy;
    vo.x = vbi.x + dt * up.x;
    vo.y = vbi.y + dt * up.y;
    ao.x = hdt * vbi.x + hdt * dt * up.x;
    ao.y = hdt * vbi.y + hdt * dt * up.y;
    A.ub_out[i] = up;
    A.vb_out[i] = vo;
    A.ab_out[i] = ao;
    A.db[i] = (P.flags[i] & kNotch) ? R(0) : A.dbn[i] + dsum;
  }
  __shared__ bool last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(P.ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    *P.ticket = 0;
    *A.kdec -= 1;
  }
}

}  // namespace pff
