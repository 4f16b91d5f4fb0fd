// Quasi-static staggered mode (Sec. 3.5; the matrix-free operator of
// Sec. 2.3): per load increment the prescribed displacement is put on the
// loaded dofs, the mechanics f_int(u; d) = 0 on the free dofs is solved by
// Newton iterations whose linear systems K_T(u) du = -r are solved by Jacobi
// PCG with the matrix-free tangent action (Eq. matrix_free_tangent_action:
// the directional derivative of the internal force, element by element
// through the split's tangent, gathered per node), then the history and
// the damage solve follow as in a dynamic step.
#pragma once
#include "adjoint.cuh"

namespace pff {

// bc flags per node: u_x fixed (to 0), u_y fixed (to 0), loaded (u_y = U).
enum : uint8_t { kQsFixX = 1, kQsFixY = 2, kQsLoaded = 4 };

struct QsScalars {
  double rr, rr0, fsq, reaction;  // |r_free|^2, |r_0|^2 of the CG, |f_int|^2 (all dofs), sum f_y (loaded)
  double rho, pq, alpha, beta;
  int32_t iters, done, status, pad;
  float alpha_f, beta_f;
};

template <typename R> struct QsParams {
  typedef typename Params<R>::R2 R2;
  typedef typename Params<R>::R4 R4;
  Params<R> P;        // mesh, material, u, d (P.u is the displacement)
  const uint8_t *bc;  // N flags
  double U;           // prescribed u_y of the loaded nodes
  R4 *pz;             // (p_x, z_x, p_y, z_y) per node
  R2 *r, *q, *x, *dg; // residual, K_T p, the Newton step, Jacobi diagonal
  R *ke;              // per element the 6 x 6 tangent K_e = A B^T C_T B (row-major,
                      // dofs (x0, y0, x1, y1, x2, y2)), rebuilt each Newton step
  QsScalars *qs;
  double tol;         // CG: |r| <= tol |r_0|
  int32_t max_it;
};

template <typename R> __device__ __forceinline__ bool qs_fx(const QsParams<R> &Q, int i) {
  return Q.bc[i] & kQsFixX;
}
template <typename R> __device__ __forceinline__ bool qs_fy(const QsParams<R> &Q, int i) {
  return Q.bc[i] & (kQsFixY | kQsLoaded);
}

// Dirichlet values: fixed components 0, loaded u_y = U.
template <typename R>
__global__ void __launch_bounds__(256) k_qs_bc(QsParams<R> Q) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Q.P.N; i += gridDim.x * blockDim.x) {
    typename Params<R>::R2 u = Q.P.u[i];
    if (qs_fx(Q, i)) u.x = R(0);
    if (qs_fy(Q, i)) u.y = (Q.bc[i] & kQsLoaded) ? (R)Q.U : R(0);
    Q.P.u[i] = u;
  }
}

// Residual r = -f_int(u; d) on the free dofs (0 on fixed ones), with
// |r_free|^2, |f_int|^2 over all dofs and the reaction sum_loaded f_y;
// zeroes the Newton step x.
template <typename R>
__global__ void __launch_bounds__(256) k_qs_residual(QsParams<R> Q) {
  typedef Acc<R> AC;
  const Params<R> &P = Q.P;
  typename AC::T vals[3] = {AC::zero(), AC::zero(), AC::zero()};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.N; i += gridDim.x * blockDim.x) {
    R fx = 0, fy = 0;
    for (int k = 0; k < P.D; ++k) {
      const int en = __ldg(&P.ell[(size_t)k * P.N + i]);
      if (en < 0) continue;
      R ex, ey, psip;
      force_entry(P, en, ex, ey, psip);
      fx = radd(fx, ex);
      fy = radd(fy, ey);
    }
    typename Params<R>::R2 r;
    r.x = qs_fx(Q, i) ? R(0) : -fx;
    r.y = qs_fy(Q, i) ? R(0) : -fy;
    Q.r[i] = r;
    typename Params<R>::R2 z;
    z.x = R(0);
    z.y = R(0);
    Q.x[i] = z;
    const R s = P.rscale;
    vals[0] = AC::add(vals[0], AC::add(AC::prod(s * r.x, s * r.x), AC::prod(s * r.y, s * r.y)));
    vals[1] = AC::add(vals[1], AC::add(AC::prod(s * fx, s * fx), AC::prod(s * fy, s * fy)));
    if (Q.bc[i] & kQsLoaded) vals[2] = AC::add(vals[2], AC::prod(fy, R(1)));
  }
  __shared__ double tot[3];
  if (reduce_last<R, 3>(vals, P.part, P.ticket, tot) && threadIdx.x == 0) {
    Q.qs->rr = tot[0];
    Q.qs->fsq = tot[1];
    Q.qs->reaction = tot[2];
  }
}

// The element's tangent stress along a strain direction de:
// dsigma = g(dbar) dsigma+[de] + dsigma-[de] at the element's strain.
template <typename R>
__device__ __forceinline__ void qs_dsigma(const Params<R> &P, R exx, R eyy, R exy, R g, const R (&de)[3],
                                          R (&ds)[3]) {
  R dsp[3], dsm[3];
  split_tangent(P, exx, eyy, exy, de, dsp, dsm);
  ds[0] = g * dsp[0] + dsm[0];
  ds[1] = g * dsp[1] + dsm[1];
  ds[2] = g * dsp[2] + dsm[2];
}

// Strain of the element at node values of a field (p_new of the CG: own
// node pc, neighbours rebuilt from (p, z) with beta).
template <typename R>
__device__ __forceinline__ typename Params<R>::R2 qs_pnew(const QsParams<R> &Q, int j, R beta) {
  const typename Params<R>::R4 v = Q.pz[j];
  typename Params<R>::R2 o;
  o.x = fma(beta, v.x, v.y);
  o.y = fma(beta, v.z, v.w);
  return o;
}

// Element tangents at the current u and d (constant during the CG of a
// Newton step): column (b, c) of K_e is A B^T dsigma[B e_(b,c)] with
// dsigma = g(dbar) dsigma+ + dsigma- (the split's tangent); the Hessian of
// A psi, so K_e is symmetric.
template <typename R>
__global__ void __launch_bounds__(256) k_qs_elem_tangent(QsParams<R> Q) {
  typedef typename Params<R>::R4 R4;
  const Params<R> &P = Q.P;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < P.Ne; e += gridDim.x * blockDim.x) {
    int4 t;
    R A;
    R4 G;
    load_elem(P, e, t, A, G);
    R exx, eyy, exy;
    elem_strain(P, G, t, exx, eyy, exy);
    const R db = (P.d[t.x] + P.d[t.y] + P.d[t.z]) * (R(1) / R(3));
    const R g = (R(1) - db) * (R(1) - db) + P.eta;
    R gxs[3], gys[3];
    for (int b = 0; b < 3; ++b) slot_grad<R>(G, b, gxs[b], gys[b]);
    R *K = Q.ke + (size_t)e * 36;
    for (int b = 0; b < 3; ++b)
      for (int c = 0; c < 2; ++c) {
        const R gx = gxs[b], gy = gys[b];
        const R de[3] = {c == 0 ? gx : R(0), c == 1 ? gy : R(0), R(0.5) * (c == 0 ? gy : gx)};
        R ds[3];
        qs_dsigma(P, exx, eyy, exy, g, de, ds);
        const int col = 2 * b + c;
        for (int a = 0; a < 3; ++a) {
          K[(2 * a) * 6 + col] = A * (ds[0] * gxs[a] + ds[2] * gys[a]);
          K[(2 * a + 1) * 6 + col] = A * (ds[2] * gxs[a] + ds[1] * gys[a]);
        }
      }
  }
}

// Jacobi diagonal of K_T(u) (one unit displacement per dof through the
// tangent), z = r / diag, p = z; rho = r.z and |r_0|.
template <typename R>
__global__ void __launch_bounds__(256) k_qs_setup(QsParams<R> Q) {
  typedef Acc<R> AC;
  typedef typename Params<R>::R4 R4;
  const Params<R> &P = Q.P;
  typename AC::T vals[1] = {AC::zero()};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.N; i += gridDim.x * blockDim.x) {
    R dx = 0, dy = 0;
    for (int k = 0; k < P.D; ++k) {
      const int en = __ldg(&P.ell[(size_t)k * P.N + i]);
      if (en < 0) continue;
      const int e = en >> 2, a = en & 3;
      const R *K = Q.ke + (size_t)e * 36;
      dx = radd(dx, K[(2 * a) * 6 + 2 * a]);
      dy = radd(dy, K[(2 * a + 1) * 6 + 2 * a + 1]);
    }
    const typename Params<R>::R2 r = Q.r[i];
    typename Params<R>::R2 dg;
    dg.x = (qs_fx(Q, i) || dx == R(0)) ? R(1) : dx;
    dg.y = (qs_fy(Q, i) || dy == R(0)) ? R(1) : dy;
    Q.dg[i] = dg;
    R4 pz;
    pz.x = R(0);
    pz.y = r.x / dg.x;
    pz.z = R(0);
    pz.w = r.y / dg.y;
    Q.pz[i] = pz;
    const R s = P.rscale;
    vals[0] = AC::add(vals[0], AC::add(AC::prod(s * r.x, pz.y), AC::prod(s * r.y, pz.w)));
  }
  __shared__ double tot[1];
  if (reduce_last<R, 1>(vals, P.part, P.ticket, tot) && threadIdx.x == 0) {
    QsScalars &S = *Q.qs;
    S.rho = tot[0];
    S.rr0 = S.rr;
    S.beta = 0.0;
    S.beta_f = 0.f;
    S.iters = 0;
    S.status = 0;
    S.done = (S.rr == 0.0) ? 1 : 0;
  }
}

// q = K_T(u) p_new on the free dofs (p_new = z + beta p, rebuilt for the
// neighbours), p_new . q -> alpha.  A no-op once the solve is done.
template <typename R>
__global__ void __launch_bounds__(256) k_qs_matvec(QsParams<R> Q) {
  typedef Acc<R> AC;
  typedef typename Params<R>::R2 R2;
  typedef typename Params<R>::R4 R4;
  const Params<R> &P = Q.P;
  if (Q.qs->done) return;
  const R beta = sizeof(R) == 4 ? (R)Q.qs->beta_f : (R)Q.qs->beta;
  typename AC::T vals[1] = {AC::zero()};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.N; i += gridDim.x * blockDim.x) {
    R qx = 0, qy = 0;
    for (int k = 0; k < P.D; ++k) {
      const int en = __ldg(&P.ell[(size_t)k * P.N + i]);
      if (en < 0) continue;
      const int e = en >> 2, a = en & 3;
      const ERec<R> &rc = P.rec[e];
      const R2 p0 = qs_pnew(Q, rc.n0, beta), p1 = qs_pnew(Q, rc.n1, beta), p2 = qs_pnew(Q, rc.n2, beta);
      const R *K = Q.ke + (size_t)e * 36 + 12 * a;  // rows 2a, 2a+1
      qx = radd(qx, K[0] * p0.x + K[1] * p0.y + K[2] * p1.x + K[3] * p1.y + K[4] * p2.x + K[5] * p2.y);
      qy = radd(qy, K[6] * p0.x + K[7] * p0.y + K[8] * p1.x + K[9] * p1.y + K[10] * p2.x + K[11] * p2.y);
    }
    if (qs_fx(Q, i)) qx = R(0);
    if (qs_fy(Q, i)) qy = R(0);
    R2 q;
    q.x = qx;
    q.y = qy;
    Q.q[i] = q;
    const R2 pn = qs_pnew(Q, i, beta);
    const R s = P.rscale;
    vals[0] = AC::add(vals[0], AC::add(AC::prod(pn.x, s * qx), AC::prod(pn.y, s * qy)));
  }
  __shared__ double tot[1];
  if (reduce_last<R, 1>(vals, P.part, P.ticket, tot) && threadIdx.x == 0) {
    QsScalars &S = *Q.qs;
    S.pq = tot[0];
    S.alpha = tot[0] != 0.0 ? S.rho / tot[0] : 0.0;
    S.alpha_f = (float)S.alpha;
  }
}

// x += alpha p, r -= alpha q, z = r / diag, (p, z) stored; |r|^2, r.z ->
// beta and the stop test |r| <= tol |r_0|.
template <typename R>
__global__ void __launch_bounds__(256) k_qs_update(QsParams<R> Q) {
  typedef Acc<R> AC;
  typedef typename Params<R>::R2 R2;
  typedef typename Params<R>::R4 R4;
  const Params<R> &P = Q.P;
  if (Q.qs->done) return;
  const R beta = sizeof(R) == 4 ? (R)Q.qs->beta_f : (R)Q.qs->beta;
  const R alpha = sizeof(R) == 4 ? (R)Q.qs->alpha_f : (R)Q.qs->alpha;
  typename AC::T vals[2] = {AC::zero(), AC::zero()};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.N; i += gridDim.x * blockDim.x) {
    const R2 pn = qs_pnew(Q, i, beta), q = Q.q[i], dg = Q.dg[i];
    R2 x = Q.x[i], r = Q.r[i];
    x.x = fma(alpha, pn.x, x.x);
    x.y = fma(alpha, pn.y, x.y);
    r.x = fma(-alpha, q.x, r.x);
    r.y = fma(-alpha, q.y, r.y);
    if (qs_fx(Q, i)) r.x = R(0);
    if (qs_fy(Q, i)) r.y = R(0);
    Q.x[i] = x;
    Q.r[i] = r;
    R4 pz;
    pz.x = pn.x;
    pz.y = r.x / dg.x;
    pz.z = pn.y;
    pz.w = r.y / dg.y;
    Q.pz[i] = pz;
    const R s = P.rscale;
    vals[0] = AC::add(vals[0], AC::add(AC::prod(s * r.x, s * r.x), AC::prod(s * r.y, s * r.y)));
    vals[1] = AC::add(vals[1], AC::add(AC::prod(s * r.x, pz.y), AC::prod(s * r.y, pz.w)));
  }
  __shared__ double tot[2];
  if (reduce_last<R, 2>(vals, P.part, P.ticket, tot) && threadIdx.x == 0) {
    QsScalars &S = *Q.qs;
    S.iters += 1;
    S.rr = tot[0];
    if (!(tot[0] == tot[0]) || isinf(tot[0])) {
      S.status = kStNonfinite;
      S.done = 1;
    } else if (S.pq == 0.0 || sqrt(tot[0]) <= Q.tol * sqrt(S.rr0)) {
      S.done = 1;
    } else if (S.iters >= Q.max_it) {
      S.status = kStNotConverged;
      S.done = 1;
    }
    S.beta = S.rho != 0.0 ? tot[1] / S.rho : 0.0;
    S.beta_f = (float)S.beta;
    S.rho = tot[1];
  }
}

// u += x on the free dofs.
template <typename R>
__global__ void __launch_bounds__(256) k_qs_apply(QsParams<R> Q) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Q.P.N; i += gridDim.x * blockDim.x) {
    typename Params<R>::R2 u = Q.P.u[i];
    const typename Params<R>::R2 x = Q.x[i];
    if (!qs_fx(Q, i)) u.x += x.x;
    if (!qs_fy(Q, i)) u.y += x.y;
    Q.P.u[i] = u;
  }
}

// History H = max(H, psi+(u)) per element (the owner-entry rule of the
// dynamic step, element by element).
template <typename R>
__global__ void __launch_bounds__(256) k_qs_history(QsParams<R> Q) {
  typedef typename Params<R>::R4 R4;
  const Params<R> &P = Q.P;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < P.Ne; e += gridDim.x * blockDim.x) {
    int4 t;
    R A;
    R4 G;
    load_elem(P, e, t, A, G);
    R exx, eyy, exy;
    elem_strain(P, G, t, exx, eyy, exy);
    R sxx, syy, sxy, psip;
    stress(P, exx, eyy, exy, R(1), sxx, syy, sxy, psip);
    history_update(P, e << 2, psip);
  }
}

}  // namespace pff
