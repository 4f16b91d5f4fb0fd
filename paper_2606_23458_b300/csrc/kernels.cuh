// kernels.cuh -- device code of the phase-field fracture step for sm_103a.
//
// Every node-indexed kernel runs one thread per node and walks that node's
// incident elements (the node-to-element incidence, ascending element id),
// recomputing what it needs of each element.  Accumulation is therefore a
// plain per-thread sum in a fixed order: no atomics, bit-identical reruns.
// Per-element results that must be stored once (the history H, the damage
// mass coefficient) are written by the element's slot-0 node ("owner").
//
// Reductions (CG inner products, energies) are FP64: each block reduces with
// warp shuffles, writes one partial per block, and the last block to finish
// (ticket counter) sums the partials in block order.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace pff {

enum : int { kSpectral = 0, kAmor = 1, kIso = 2 };
enum : int { kAT1 = 1, kAT2 = 2 };
enum : uint8_t { kNotch = 1, kLoaded = 2 };
enum : int { kStOk = 0, kStNotConverged = 5, kStTimeout = 6, kStNonfinite = 7 };

template <typename R> struct V;
template <> struct V<float> {
  typedef float2 T2;
  typedef float4 T4;
};
struct __align__(16) dbl4 { double x, y, z, w; };
template <> struct V<double> {
  typedef double2 T2;
  typedef dbl4 T4;
};

// Scalars of one damage solve, living in device memory.
struct SolveScalars {
  double bn;      // ||b - A 1_D|| over free rows
  double rho;     // r . z
  double alpha, beta;
  double rr;      // ||r||^2 (free rows)
  double pq;
  int32_t iters, restarts, status, done;
  int32_t projected, inner_done, pad0, pad1;
};

// Everything a kernel needs, passed by value (graph-captured).
template <typename R> struct Params {
  typedef typename V<R>::T2 R2;
  typedef typename V<R>::T4 R4;
  int32_t N, Ne;
  // mesh
  const int32_t *__restrict__ ptr;
  const int32_t *__restrict__ ent;
  const int4 *__restrict__ tri;
  const R4 *__restrict__ grad;   // (dphi0/dx, dphi0/dy, dphi1/dx, dphi1/dy)
  const R *__restrict__ area;
  const uint8_t *__restrict__ flags;
  const R2 *__restrict__ fext;
  const R *__restrict__ minv;
  // material
  R lam, mu, K, eta;
  int32_t split, model;
  R kappa;      // damage diffusion coefficient (Gc l0 or 3/4 Gc l0)
  double cbase; // reaction: c_e = cbase + 2 H_e
  double wbase; // load:     w_e = wbase + 2 H_e
  double Gc, l0;
  // state
  R2 *u, *v, *a;
  R *d;
  double *H;
  // time
  double dt, t_ramp, t_next; // t_next used when step_ctr == nullptr
  const int64_t *step_ctr;   // device step counter n (t_next = (n+1) dt)
  // damage solve
  const R *dprev;
  R *dout;
  double *x, *r, *b;
  R *z, *p, *q, *dinv, *mcoef;
  uint8_t *freef;
  double *part;
  unsigned int *ticket;
  SolveScalars *sc;
  double tol;
  int32_t max_it, max_restarts;
  int32_t use_cond;
  cudaGraphConditionalHandle cond_inner, cond_outer;
  // logs
  int32_t *iters_log;     // device, per step (iters, restarts)
  int32_t *status_word;   // device, worst status (atomicMax)
  int64_t *step_inc;      // counter incremented at the end of a step
  double *energy_out;     // 4 doubles: E_el, E_kin, E_frac, W_ext
  double *wext;           // running external work
  int32_t track_work;
};

// --------------------------------------------------------------- helpers

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Block-reduces NV doubles, publishes one partial per block and returns
// true in every thread of the last block to arrive; that block then finds
// the totals in `tot` (shared, valid after the call).  Fixed summation order.
template <int NV>
__device__ __forceinline__ bool reduce_last(const double (&v)[NV], double *part,
                                            unsigned int *ticket, double *tot) {
  __shared__ double sh[32][NV];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double s = warp_sum(v[k]);
    if (lane == 0) sh[wid][k] = s;
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double s = lane < nw ? sh[lane][k] : 0.0;
      s = warp_sum(s);
      if (lane == 0) part[(size_t)blockIdx.x * NV + k] = s;
    }
    if (lane == 0) {
      __threadfence();
      unsigned int t = atomicAdd(ticket, 1u);
      last = (t == gridDim.x - 1);
    }
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  // the last block: sum the partials in block order, strided by thread
  double acc[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) acc[k] = 0.0;
  for (int j = threadIdx.x; j < (int)gridDim.x; j += blockDim.x)
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] += __ldcg(&part[(size_t)j * NV + k]);
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double s = warp_sum(acc[k]);
    if (lane == 0) sh[wid][k] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 0; k < NV; ++k) {
      double s = 0.0;
      for (int w = 0; w < nw; ++w) s += sh[w][k];
      tot[k] = s;
    }
    *ticket = 0u;
  }
  __syncthreads();
  return true;
}

template <typename R> __device__ __forceinline__ R rpos(R x) { return x > R(0) ? x : R(0); }
template <typename R> __device__ __forceinline__ R rneg(R x) { return x < R(0) ? x : R(0); }

// Smooth traction ramp, Eq. (smooth_traction_ramp).
__device__ __forceinline__ double ramp(double t, double tr) {
  if (t <= 0.0) return 0.0;
  if (t >= tr) return 1.0;
  return 0.5 * (1.0 - cos(3.14159265358979323846 * t / tr));
}

template <typename R>
__device__ __forceinline__ double step_time(const Params<R> &P) {
  return P.step_ctr ? (double)(*P.step_ctr + 1) * P.dt : P.t_next;
}

// Degraded stress and psi+ at one element (tensor strain components).
// Spectral (Eq. spectral_split): with D = eps - tr/2 I and R = |D|, the
// tensile part is eps+ = (<e1>+ + <e2>+)/2 I + (<e1>+ - <e2>+)/(2R) D.
// Volumetric-deviatoric (Eq. amor_split) uses the 3-D deviator of the
// plane-strain tensor.  sigma = g sigma+ + sigma-.
template <typename R>
__device__ __forceinline__ void stress(const Params<R> &P, R exx, R eyy, R exy, R g,
                                       R &sxx, R &syy, R &sxy, R &psip) {
  const R tr = exx + eyy;
  const R trp = rpos(tr), trm = rneg(tr);
  if (P.split == kSpectral) {
    const R half = R(0.5) * (exx - eyy);
    const R rad = sqrt(half * half + exy * exy);
    const R e1 = R(0.5) * tr + rad, e2 = R(0.5) * tr - rad;
    const R e1p = rpos(e1), e2p = rpos(e2);
    const R s = rad > R(0) ? (e1p - e2p) / (R(2) * rad) : R(0);
    const R m = R(0.5) * (e1p + e2p);
    const R pxx = m + s * half, pyy = m - s * half, pxy = s * exy;
    const R tm = P.lam * trm, tp = P.lam * trp, mu2 = R(2) * P.mu;
    sxx = g * (tp + mu2 * pxx) + tm + mu2 * (exx - pxx);
    syy = g * (tp + mu2 * pyy) + tm + mu2 * (eyy - pyy);
    sxy = g * (mu2 * pxy) + mu2 * (exy - pxy);
    psip = R(0.5) * P.lam * trp * trp + P.mu * (e1p * e1p + e2p * e2p);
  } else if (P.split == kAmor) {
    const R t3 = tr * (R(1) / R(3)), mu2 = R(2) * P.mu;
    sxx = g * (P.K * trp + mu2 * (exx - t3)) + P.K * trm;
    syy = g * (P.K * trp + mu2 * (eyy - t3)) + P.K * trm;
    sxy = g * (mu2 * exy);
    psip = R(0.5) * P.K * trp * trp +
           P.mu * (exx * exx + eyy * eyy + R(2) * exy * exy - tr * t3);
  } else {
    const R mu2 = R(2) * P.mu;
    sxx = g * (P.lam * tr + mu2 * exx);
    syy = g * (P.lam * tr + mu2 * eyy);
    sxy = g * (mu2 * exy);
    psip = R(0.5) * P.lam * tr * tr + P.mu * (exx * exx + eyy * eyy + R(2) * exy * exy);
  }
}

template <typename R, typename R4>
__device__ __forceinline__ void slot_grad(const R4 &G, int a, R &gx, R &gy) {
  gx = a == 0 ? G.x : (a == 1 ? G.z : -(G.x + G.z));
  gy = a == 0 ? G.y : (a == 1 ? G.w : -(G.y + G.w));
}

// ------------------------------------------------------------ mechanics

// Predictor, Eq. (vv_u): u += dt v + dt^2/2 a.  With track_work the
// trapezoid-rule external work increment 1/2 (S_n + S_n+1) f_ext . du is
// reduced into *wext.
template <typename R>
__global__ void k_predict(Params<R> P) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double w = 0.0;
  if (i < P.N) {
    typename Params<R>::R2 u = P.u[i], v = P.v[i], a = P.a[i];
    const R dt = (R)P.dt, h = R(0.5) * dt * dt;
    const R dux = dt * v.x + h * a.x, duy = dt * v.y + h * a.y;
    if (P.track_work && (P.flags[i] & kLoaded)) {
      const double t1 = step_time(P), t0 = t1 - P.dt;
      const double S = 0.5 * (ramp(t0, P.t_ramp) + ramp(t1, P.t_ramp));
      typename Params<R>::R2 f = P.fext[i];
      w = S * ((double)f.x * dux + (double)f.y * duy);
    }
    u.x += dux;
    u.y += duy;
    P.u[i] = u;
  }
  if (P.track_work) {
    double v1[1] = {w};
    __shared__ double tot[1];
    if (reduce_last<1>(v1, P.part, P.ticket, tot) && threadIdx.x == 0) *P.wext += tot[0];
  }
}

// Internal force at u_{n+1} with d_n, history update, Eqs. (vv_a), (vv_v).
template <typename R>
__global__ void __launch_bounds__(256) k_force(Params<R> P) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P.N) return;
  typedef typename Params<R>::R2 R2;
  typedef typename Params<R>::R4 R4;
  R fx = 0, fy = 0;
  const int k0 = P.ptr[i], k1 = P.ptr[i + 1];
  for (int k = k0; k < k1; ++k) {
    const int en = __ldg(&P.ent[k]);
    const int e = en >> 2, a = en & 3;
    const int4 t = __ldg(&P.tri[e]);
    const R4 G = P.grad[e];
    const R A = __ldg(&P.area[e]);
    const R2 u0 = P.u[t.x], u1 = P.u[t.y], u2 = P.u[t.z];
    const R d0 = P.d[t.x], d1 = P.d[t.y], d2 = P.d[t.z];
    const R ax0 = u0.x - u2.x, ax1 = u1.x - u2.x, ay0 = u0.y - u2.y, ay1 = u1.y - u2.y;
    const R exx = G.x * ax0 + G.z * ax1;
    const R eyy = G.y * ay0 + G.w * ay1;
    const R exy = R(0.5) * (G.y * ax0 + G.w * ax1 + G.x * ay0 + G.z * ay1);
    const R db = (d0 + d1 + d2) * (R(1) / R(3));
    const R g = (R(1) - db) * (R(1) - db) + P.eta;
    R sxx, syy, sxy, psip;
    stress(P, exx, eyy, exy, g, sxx, syy, sxy, psip);
    R gx, gy;
    slot_grad<R>(G, a, gx, gy);
    fx += A * (sxx * gx + sxy * gy);
    fy += A * (sxy * gx + syy * gy);
    if (a == 0) {
      const double hp = (double)psip;
      if (hp > P.H[e]) P.H[e] = hp;
    }
  }
  const uint8_t fl = P.flags[i];
  R S = 0, fex = 0, fey = 0;
  if (fl & kLoaded) {
    S = (R)ramp(step_time(P), P.t_ramp);
    const R2 fe = P.fext[i];
    fex = fe.x;
    fey = fe.y;
  }
  const R mi = P.minv[i];
  const R anx = mi * (S * fex - fx), any = mi * (S * fey - fy);
  R2 v = P.v[i], ao = P.a[i];
  const R hd = R(0.5) * (R)P.dt;
  v.x += hd * (ao.x + anx);
  v.y += hd * (ao.y + any);
  P.v[i] = v;
  R2 an;
  an.x = anx;
  an.y = any;
  P.a[i] = an;
}

// --------------------------------------------------------------- damage

// Right-hand side, Jacobi diagonal, lifted initial residual and mass
// coefficients of the damage problem (AT2: Eq. damage_pde_at2; AT1: Eq.
// damage_pde_at1), consistent mass M^e = A_e (1 + delta_ab)/12.
//   x0 = d_prev (1 on the notch), r = b - A x0, b_eff = b - A 1_D.
template <typename R>
__global__ void __launch_bounds__(256) k_dmg_rhs(Params<R> P) {
  typedef typename Params<R>::R4 R4;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double vals[3] = {0.0, 0.0, 0.0};  // |b_eff|^2, |r|^2, r.z
  if (i < P.N) {
    const bool notch = P.flags[i] & kNotch;
    double bi = 0, dg = 0, ax = 0, a1 = 0;
    const int k0 = P.ptr[i], k1 = P.ptr[i + 1];
    for (int k = k0; k < k1; ++k) {
      const int en = __ldg(&P.ent[k]);
      const int e = en >> 2, a = en & 3;
      const int4 t = __ldg(&P.tri[e]);
      const R4 G = P.grad[e];
      const double A = (double)__ldg(&P.area[e]);
      const double h = P.H[e];
      const double c = P.cbase + 2.0 * h, w = P.wbase + 2.0 * h;
      if (a == 0) P.mcoef[e] = (R)(c * A / 12.0);
      if (notch) continue;
      const bool n0 = P.flags[t.x] & kNotch, n1 = P.flags[t.y] & kNotch, n2 = P.flags[t.z] & kNotch;
      const double x0 = n0 ? 1.0 : (double)P.dprev[t.x];
      const double x1 = n1 ? 1.0 : (double)P.dprev[t.y];
      const double x2 = n2 ? 1.0 : (double)P.dprev[t.z];
      const double o0 = n0 ? 1.0 : 0.0, o1 = n1 ? 1.0 : 0.0, o2 = n2 ? 1.0 : 0.0;
      R gxr, gyr;
      slot_grad<R>(G, a, gxr, gyr);
      const double gx = gxr, gy = gyr;
      const double G0x = G.x, G0y = G.y, G1x = G.z, G1y = G.w;
      const double kA = (double)P.kappa * A, mA = c * A / 12.0;
      bi += w * A / 3.0;
      dg += kA * (gx * gx + gy * gy) + 2.0 * mA;
      const double xa = a == 0 ? x0 : (a == 1 ? x1 : x2);
      const double oa = a == 0 ? o0 : (a == 1 ? o1 : o2);
      ax += kA * (gx * (G0x * (x0 - x2) + G1x * (x1 - x2)) + gy * (G0y * (x0 - x2) + G1y * (x1 - x2))) +
            mA * (xa + x0 + x1 + x2);
      a1 += kA * (gx * (G0x * (o0 - o2) + G1x * (o1 - o2)) + gy * (G0y * (o0 - o2) + G1y * (o1 - o2))) +
            mA * (oa + o0 + o1 + o2);
    }
    if (notch) {
      P.x[i] = 1.0;
      P.r[i] = 0.0;
      P.z[i] = R(0);
      P.p[i] = R(0);
      P.dinv[i] = R(0);
      if (P.b) P.b[i] = 0.0;
    } else {
      const double x0 = (double)P.dprev[i];
      const double ri = bi - ax, be = bi - a1;
      const double di = 1.0 / dg;
      const R zi = (R)(ri * di);
      P.x[i] = x0;
      P.r[i] = ri;
      P.dinv[i] = (R)di;
      P.z[i] = zi;
      P.p[i] = R(0);
      if (P.b) P.b[i] = bi;
      vals[0] = be * be;
      vals[1] = ri * ri;
      vals[2] = ri * (double)zi;
    }
  }
  __shared__ double tot[3];
  if (reduce_last<3>(vals, P.part, P.ticket, tot) && threadIdx.x == 0) {
    SolveScalars &S = *P.sc;
    S.bn = sqrt(tot[0]);
    S.rr = tot[1];
    S.rho = tot[2];
    S.beta = 0.0;
    S.alpha = 0.0;
    S.iters = 0;
    S.restarts = 0;
    S.status = kStOk;
    S.projected = 0;
    const bool done = (P.model == kAT2) && (S.bn == 0.0 || sqrt(S.rr) <= P.tol * S.bn);
    S.done = done ? 1 : 0;
    if (P.use_cond) cudaGraphSetConditional(P.cond_inner, done ? 0u : 1u);
  }
}

// Value of the next search direction at node j: p_new = z + beta p_old
// (zero on the notch and, for AT1, outside the free set).
template <typename R>
__device__ __forceinline__ R pnew(const Params<R> &P, int j, R beta) {
  return fma(beta, P.p[j], P.z[j]);
}

// q = A p_new on free rows (matrix-free, Eq. matrix_free_fe_operator), and
// the reduction p_new . q -> alpha = rho / (p.q).
template <typename R>
__global__ void __launch_bounds__(256) k_cg_matvec(Params<R> P) {
  typedef typename Params<R>::R4 R4;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double vals[1] = {0.0};
  const R beta = (R)P.sc->beta;
  if (i < P.N) {
    const bool fixed = (P.flags[i] & kNotch) || (P.freef && !P.freef[i]);
    if (!fixed) {
      R q = 0;
      const int k0 = P.ptr[i], k1 = P.ptr[i + 1];
      for (int k = k0; k < k1; ++k) {
        const int en = __ldg(&P.ent[k]);
        const int e = en >> 2, a = en & 3;
        const int4 t = __ldg(&P.tri[e]);
        const R4 G = P.grad[e];
        const R kA = P.kappa * __ldg(&P.area[e]);
        const R mc = P.mcoef[e];
        const R p0 = pnew(P, t.x, beta), p1 = pnew(P, t.y, beta), p2 = pnew(P, t.z, beta);
        const R dx = G.x * (p0 - p2) + G.z * (p1 - p2);
        const R dy = G.y * (p0 - p2) + G.w * (p1 - p2);
        R gx, gy;
        slot_grad<R>(G, a, gx, gy);
        const R pa = a == 0 ? p0 : (a == 1 ? p1 : p2);
        q += kA * (gx * dx + gy * dy) + mc * (pa + p0 + p1 + p2);
      }
      P.q[i] = q;
      vals[0] = (double)pnew(P, i, beta) * (double)q;
    } else {
      P.q[i] = R(0);
    }
  }
  __shared__ double tot[1];
  if (reduce_last<1>(vals, P.part, P.ticket, tot) && threadIdx.x == 0) {
    SolveScalars &S = *P.sc;
    S.pq = tot[0];
    S.alpha = tot[0] != 0.0 ? S.rho / tot[0] : 0.0;
  }
}

// x += alpha p, r -= alpha q, z = r / diag, p = p_new; reductions |r|^2 and
// r.z; the last block takes the stop decision (Sec. 2.4; stop test on the
// unpreconditioned residual).  AT1 (lo = d_prev, hi = 1): values leaving
// the box are projected and flag a restart.
template <typename R>
__global__ void __launch_bounds__(256) k_cg_update(Params<R> P) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double vals[3] = {0.0, 0.0, 0.0};
  const R beta = (R)P.sc->beta;
  const double alpha = P.sc->alpha;
  if (i < P.N) {
    const bool fixed = (P.flags[i] & kNotch) || (P.freef && !P.freef[i]);
    if (!fixed) {
      const R pn = pnew(P, i, beta);
      double xi = P.x[i] + alpha * (double)pn;
      const double ri = P.r[i] - alpha * (double)P.q[i];
      if (P.model == kAT1) {
        const double lo = (double)P.dprev[i];
        if (xi < lo) { xi = lo; vals[2] = 1.0; }
        if (xi > 1.0) { xi = 1.0; vals[2] = 1.0; }
      }
      const R zi = (R)(ri * (double)P.dinv[i]);
      P.x[i] = xi;
      P.r[i] = ri;
      P.z[i] = zi;
      P.p[i] = pn;
      vals[0] = ri * ri;
      vals[1] = ri * (double)zi;
    }
  }
  __shared__ double tot[3];
  if (reduce_last<3>(vals, P.part, P.ticket, tot) && threadIdx.x == 0) {
    SolveScalars &S = *P.sc;
    S.iters += 1;
    S.rr = tot[0];
    const double rz = tot[1];
    bool stop = false;
    if (!(tot[0] == tot[0]) || isinf(tot[0])) {
      S.status = kStNonfinite;
      S.done = 1;
      stop = true;
    } else if (P.model == kAT1 && tot[2] > 0.0) {
      S.projected = 1;
      stop = true;  // restart
    } else if (sqrt(tot[0]) <= P.tol * S.bn) {
      if (P.model == kAT2) S.done = 1;
      stop = true;
    } else if (S.pq == 0.0) {
      if (P.model == kAT2) S.done = 1;
      stop = true;
    }
    if (!stop && S.iters >= P.max_it) {
      S.status = kStNotConverged;
      S.done = 1;
      stop = true;
    }
    S.beta = S.rho != 0.0 ? rz / S.rho : 0.0;
    S.rho = rz;
    S.inner_done = stop ? 1 : 0;
    if (P.use_cond) cudaGraphSetConditional(P.cond_inner, stop ? 0u : 1u);
  }
}

// AT1 restart (projected CG, Sec. 2.4): r = b - A x, active set
// {x <= lo, r <= 0} U {x >= hi, r >= 0}, free-set residual norm, a fresh
// direction p = z; converged when ||r_F|| <= tol ||b_eff||.
template <typename R>
__global__ void __launch_bounds__(256) k_at1_restart(Params<R> P) {
  typedef typename Params<R>::R4 R4;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double vals[2] = {0.0, 0.0};
  if (i < P.N) {
    const bool notch = P.flags[i] & kNotch;
    if (!notch) {
      double ax = 0;
      const int k0 = P.ptr[i], k1 = P.ptr[i + 1];
      for (int k = k0; k < k1; ++k) {
        const int en = __ldg(&P.ent[k]);
        const int e = en >> 2, a = en & 3;
        const int4 t = __ldg(&P.tri[e]);
        const R4 G = P.grad[e];
        const double A = (double)__ldg(&P.area[e]);
        const double c = P.cbase + 2.0 * P.H[e];
        const double x0 = __ldcg(&P.x[t.x]), x1 = __ldcg(&P.x[t.y]), x2 = __ldcg(&P.x[t.z]);
        R gxr, gyr;
        slot_grad<R>(G, a, gxr, gyr);
        const double gx = gxr, gy = gyr;
        const double kA = (double)P.kappa * A, mA = c * A / 12.0;
        const double xa = a == 0 ? x0 : (a == 1 ? x1 : x2);
        ax += kA * (gx * ((double)G.x * (x0 - x2) + (double)G.z * (x1 - x2)) +
                    gy * ((double)G.y * (x0 - x2) + (double)G.w * (x1 - x2))) +
              mA * (xa + x0 + x1 + x2);
      }
      const double xi = P.x[i], ri = P.b[i] - ax, lo = (double)P.dprev[i];
      const bool act = (xi <= lo && ri <= 0.0) || (xi >= 1.0 && ri >= 0.0);
      P.r[i] = ri;
      P.freef[i] = act ? 0 : 1;
      P.p[i] = R(0);
      if (act) {
        P.z[i] = R(0);
      } else {
        const R zi = (R)(ri * (double)P.dinv[i]);
        P.z[i] = zi;
        vals[0] = ri * ri;
        vals[1] = ri * (double)zi;
      }
    } else {
      P.freef[i] = 0;
    }
  }
  __shared__ double tot[2];
  if (reduce_last<2>(vals, P.part, P.ticket, tot) && threadIdx.x == 0) {
    SolveScalars &S = *P.sc;
    S.rr = tot[0];
    S.rho = tot[1];
    S.beta = 0.0;
    S.projected = 0;
    bool conv = sqrt(tot[0]) <= P.tol * S.bn;
    bool stop = conv;
    if (!conv && (S.restarts >= P.max_restarts || S.iters >= P.max_it)) {
      S.status = kStNotConverged;
      stop = true;
    }
    if (!(tot[0] == tot[0])) {
      S.status = kStNonfinite;
      stop = true;
    }
    if (!stop) S.restarts += 1;
    S.done = stop ? 1 : 0;
    S.inner_done = stop ? 1 : 0;
    if (P.use_cond) {
      cudaGraphSetConditional(P.cond_outer, stop ? 0u : 1u);
      cudaGraphSetConditional(P.cond_inner, stop ? 0u : 1u);
    }
  }
}

// End of the solve: AT2 clamp d = min(1, max(x, d_prev)) (Sec. 2.4), AT1
// d = x; notch d = 1.  Logs the iteration count and status of the step and
// advances the step counter.
template <typename R>
__global__ void k_dmg_finish(Params<R> P) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < P.N) {
    double v;
    if (P.flags[i] & kNotch) {
      v = 1.0;
    } else {
      v = P.x[i];
      if (P.model == kAT2) {
        const double lo = (double)P.dprev[i];
        v = v > lo ? v : lo;
        v = v < 1.0 ? v : 1.0;
      }
    }
    P.dout[i] = (R)v;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const SolveScalars &S = *P.sc;
    if (P.status_word && S.status) atomicMax(P.status_word, S.status);
    if (P.iters_log && P.step_ctr) {
      const int64_t n = *P.step_ctr;
      P.iters_log[2 * n] = S.iters;
      P.iters_log[2 * n + 1] = S.restarts;
    }
    if (P.step_inc) *P.step_inc += 1;
  }
}

// ------------------------------------------------------------- energies

// E_el = sum A_e (g psi+ + psi-), E_frac per model, E_kin = 1/2 sum m v^2.
// Element terms are counted by the owner node (slot 0).
template <typename R>
__global__ void __launch_bounds__(256) k_energies(Params<R> P) {
  typedef typename Params<R>::R2 R2;
  typedef typename Params<R>::R4 R4;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double vals[3] = {0.0, 0.0, 0.0};
  if (i < P.N) {
    const R2 vi = P.v[i];
    vals[1] = 0.5 / (double)P.minv[i] * ((double)vi.x * vi.x + (double)vi.y * vi.y);
    const int k0 = P.ptr[i], k1 = P.ptr[i + 1];
    for (int k = k0; k < k1; ++k) {
      const int en = __ldg(&P.ent[k]);
      if (en & 3) continue;
      const int e = en >> 2;
      const int4 t = __ldg(&P.tri[e]);
      const R4 G = P.grad[e];
      const double A = (double)__ldg(&P.area[e]);
      const R2 u0 = P.u[t.x], u1 = P.u[t.y], u2 = P.u[t.z];
      const R ax0 = u0.x - u2.x, ax1 = u1.x - u2.x, ay0 = u0.y - u2.y, ay1 = u1.y - u2.y;
      const R exx = G.x * ax0 + G.z * ax1;
      const R eyy = G.y * ay0 + G.w * ay1;
      const R exy = R(0.5) * (G.y * ax0 + G.w * ax1 + G.x * ay0 + G.z * ay1);
      const double d0 = P.d[t.x], d1 = P.d[t.y], d2 = P.d[t.z];
      const double db = (d0 + d1 + d2) / 3.0;
      const double g = (1.0 - db) * (1.0 - db) + (double)P.eta;
      // psi = g psi+ + psi-: evaluate the split at g and at g = 0 via the
      // stress; psi- = psi_full - psi+ for all three splits.
      R sxx, syy, sxy, psip;
      stress(P, exx, eyy, exy, R(1), sxx, syy, sxy, psip);
      const double tr = (double)exx + eyy;
      const double full = 0.5 * (double)P.lam * tr * tr +
                          (double)P.mu * ((double)exx * exx + (double)eyy * eyy + 2.0 * (double)exy * exy);
      const double psim = P.split == kIso ? 0.0 : full - (double)psip;
      vals[0] += A * (g * (double)psip + psim);
      const double G0x = G.x, G0y = G.y, G1x = G.z, G1y = G.w;
      const double gdx = G0x * (d0 - d2) + G1x * (d1 - d2);
      const double gdy = G0y * (d0 - d2) + G1y * (d1 - d2);
      const double g2 = gdx * gdx + gdy * gdy;
      if (P.model == kAT1) {
        vals[2] += P.Gc * 0.375 * (A / 3.0 * (d0 + d1 + d2) / P.l0 + P.l0 * A * g2);
      } else {
        const double dMd = A / 12.0 * (2.0 * (d0 * d0 + d1 * d1 + d2 * d2) + 2.0 * (d0 * d1 + d1 * d2 + d0 * d2));
        vals[2] += P.Gc * (dMd / (2.0 * P.l0) + 0.5 * P.l0 * A * g2);
      }
    }
  }
  __shared__ double tot[3];
  if (reduce_last<3>(vals, P.part, P.ticket, tot) && threadIdx.x == 0) {
    P.energy_out[0] = tot[0];
    P.energy_out[1] = tot[1];
    P.energy_out[2] = tot[2];
    P.energy_out[3] = P.wext ? *P.wext : 0.0;
  }
}

}  // namespace pff
