// Quasi-static staggered mode (Sec. 3.5; the matrix-free operator of
// Sec. 2.3): per load increment the prescribed displacement is put on the
// loaded dofs, the mechanics f_int(u; d) = 0 on the free dofs is solved by
// Newton iterations whose linear systems K_T(u) du = -r are solved by Jacobi
// PCG with the matrix-free tangent action (Eq. matrix_free_tangent_action:
// the directional derivative of the internal force, element by element
// through the split's tangent, gathered per node), then the history and
// the damage solve follow as in a dynamic step.
//
// Two precisions: R, the mesh's (state u, d, H, the Newton residual, the
// element tangents' evaluation, history and damage), and K, the Krylov
// solve's (its vectors and the stored element tangents).  K = float under
// an FP64 mesh is mixed-precision iterative refinement: each Newton step
// solves in FP32 to a forcing tolerance and the FP64 residual corrects it.
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

// Per element, for the Krylov solve: node ids, the tangent T = A C_T
// (row-major 3 x 3, tensor strain (e_xx, e_yy, e_xy) -> stress, times the
// area) and the shape gradients (dphi0/dx, dphi0/dy, dphi1/dx, dphi1/dy).
// 64 bytes in FP32, 128 in FP64.
template <typename K> struct QRec;
template <> struct __align__(64) QRec<float> {
  int n0, n1, n2;
  float t[9];
  float g[4];
};
template <> struct __align__(128) QRec<double> {
  int n0, n1, n2, pad;
  double g[4];
  double t[9];
};

template <typename K> struct QkParams {
  typedef typename V<K>::T2 K2;
  typedef typename V<K>::T4 K4;
  int N, D;
  const int *ell;     // incidence, ELL: entry k of node i at ell[k N + i] = (e << 2) | slot, or -1
  QRec<K> *rec;       // Ne
  const uint8_t *bc;  // N flags
  K4 *pz;             // (p_x, z_x, p_y, z_y) per node
  K2 *r, *q, *x, *dg; // residual, K_T p, the Newton step, Jacobi diagonal
  K2 *fe;             // 3 Ne: per element and slot the force A B_a^T C_T B p_e
  // FP32 entry records of the tangent (nullable; meshes whose elements span
  // fewer than 2^15 node ids): per incidence slot k of node i (at k N + i)
  // the 16-bit offsets of the entry's other two nodes b, c (packed) and the
  // 2 x 2 blocks K_ab, K_ac of the element tangent (row-major xx, xy, yx,
  // yy).  The element's rows annihilate translations (K_aa = -K_ab - K_ac),
  // so row i is sum_k K_ab (p_b - p_i) + K_ac (p_c - p_i): a rigid
  // translation gives exactly 0 in FP32 too, and no diagonal block is kept
  uint32_t *ofs;
  float4 *kb, *kc;
  // merged rows of width 6 (nullable nbk: rows with more than six distinct
  // neighbours keep the entry records): the row's ascending neighbour
  // offsets (three words, incidence-style layout w N + i), the slot map of
  // its incidence entries (one 8-byte word per row) and per neighbour slot
  // the sum of the entries' 2 x 2 blocks for that neighbour (at j N + i;
  // padding slots offset 0, block 0).  Row i is then
  // sum_j K_ij (p_j - p_i), K_ij the exact transpose of K_ji (two
  // elements per edge: the sum does not depend on their order).
  const uint32_t *nbo;
  const uint2 *nmap;
  float4 *nbk;
  // fan order of the entry records (nullable; the mesh's fan tables, see
  // Params::fno): with them kb and kc are stored by fan position, the
  // fan's k-th triangle coupling v_k and v_{k+1 mod m}, and a row gathers
  // each distinct neighbour once
  const uint32_t *fno, *fmap;
  QsScalars *qs;
  double *part;       // per-block partial sums and the ticket of reduce_last
  unsigned int *ticket;
  double tol;         // CG: |r| <= tol |r_0|
  int32_t max_it;
};

template <typename R, typename K> struct QsParams {
  Params<R> P;        // mesh, material, u, d (P.u is the displacement)
  QkParams<K> I;      // the Krylov solve
  double U;           // prescribed u_y of the loaded nodes
};

__device__ __forceinline__ bool qs_fx(const uint8_t *bc, int i) { return bc[i] & kQsFixX; }
__device__ __forceinline__ bool qs_fy(const uint8_t *bc, int i) { return bc[i] & (kQsFixY | kQsLoaded); }

// Dirichlet values: fixed components 0, loaded u_y = U.
template <typename R, typename K>
__global__ void __launch_bounds__(256) k_qs_bc(QsParams<R, K> Q) {
  const uint8_t *bc = Q.I.bc;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Q.P.N; i += gridDim.x * blockDim.x) {
    typename Params<R>::R2 u = Q.P.u[i];
    if (qs_fx(bc, i)) u.x = R(0);
    if (qs_fy(bc, i)) u.y = (bc[i] & kQsLoaded) ? (R)Q.U : R(0);
    Q.P.u[i] = u;
  }
}

// Residual r = -f_int(u; d) on the free dofs (0 on fixed ones), evaluated
// in R and stored in K, with |r_free|^2, |f_int|^2 over all dofs and the
// reaction sum_loaded f_y; zeroes the Newton step x.
template <typename R, typename K>
__global__ void __launch_bounds__(256) k_qs_residual(QsParams<R, K> Q) {
  typedef Acc<R> AC;
  const Params<R> &P = Q.P;
  const uint8_t *bc = Q.I.bc;
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
    const R rx = qs_fx(bc, i) ? R(0) : -fx, ry = qs_fy(bc, i) ? R(0) : -fy;
    typename V<K>::T2 r, z;
    r.x = (K)rx;
    r.y = (K)ry;
    z.x = K(0);
    z.y = K(0);
    Q.I.r[i] = r;
    Q.I.x[i] = z;
    vals[0] = AC::add(vals[0], AC::add(AC::prod(rx, rx), AC::prod(ry, ry)));
    vals[1] = AC::add(vals[1], AC::add(AC::prod(fx, fx), AC::prod(fy, fy)));
    if (bc[i] & kQsLoaded) vals[2] = AC::add(vals[2], AC::prod(fy, R(1)));
  }
  __shared__ double tot[3];
  if (reduce_last<R, 3>(vals, P.part, P.ticket, tot) && threadIdx.x == 0) {
    Q.I.qs->rr = tot[0];
    Q.I.qs->fsq = tot[1];
    Q.I.qs->reaction = tot[2];
  }
}

// Element tangents at the current u and d (constant during the CG of a
// Newton step): column j of C_T is dsigma[e_j] = g(dbar) dsigma+[e_j] +
// dsigma-[e_j] (the split's tangent, linear in the strain direction), for
// the unit tensor strains e_j; stored as A C_T with the gradients.
template <typename R, typename K>
__global__ void __launch_bounds__(256) k_qs_elem_tangent(QsParams<R, K> Q) {
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
    QRec<K> o;
    o.n0 = t.x;
    o.n1 = t.y;
    o.n2 = t.z;
    o.g[0] = (K)G.x;
    o.g[1] = (K)G.y;
    o.g[2] = (K)G.z;
    o.g[3] = (K)G.w;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const R de[3] = {j == 0 ? R(1) : R(0), j == 1 ? R(1) : R(0), j == 2 ? R(1) : R(0)};
      R dsp[3], dsm[3];
      split_tangent(P, exx, eyy, exy, de, dsp, dsm);
#pragma unroll
      for (int i = 0; i < 3; ++i) o.t[3 * i + j] = (K)(A * (g * dsp[i] + dsm[i]));
    }
    Q.I.rec[e] = o;
  }
}

template <typename K>
__device__ __forceinline__ void qrec_load(const QRec<K> *rp, int &n0, int &n1, int &n2, K (&t)[9], K (&g)[4]) {
  if (sizeof(K) == 4) {
    const float4 *f = reinterpret_cast<const float4 *>(rp);
    const float4 a = __ldg(f), b = __ldg(f + 1), c = __ldg(f + 2), d = __ldg(f + 3);
    n0 = __float_as_int(a.x);
    n1 = __float_as_int(a.y);
    n2 = __float_as_int(a.z);
    t[0] = a.w; t[1] = b.x; t[2] = b.y; t[3] = b.z; t[4] = b.w;
    t[5] = c.x; t[6] = c.y; t[7] = c.z; t[8] = c.w;
    g[0] = d.x; g[1] = d.y; g[2] = d.z; g[3] = d.w;
  } else {
    const int4 n = __ldg(reinterpret_cast<const int4 *>(rp));
    n0 = n.x;
    n1 = n.y;
    n2 = n.z;
    const double2 *f = reinterpret_cast<const double2 *>(rp) + 1;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const double2 v = __ldg(f + k);
      g[2 * k] = (K)v.x;
      g[2 * k + 1] = (K)v.y;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const double2 v = __ldg(f + 2 + k);
      t[2 * k] = (K)v.x;
      t[2 * k + 1] = (K)v.y;
    }
    t[8] = (K)__ldg(reinterpret_cast<const double *>(f + 6));
  }
}

// Node force of slot a from the element tangent applied to a strain:
// A B_a^T C_T de.
template <typename K>
__device__ __forceinline__ void qs_slot_force(const K (&t)[9], const K (&g)[4], int a, const K (&de)[3], K &fx,
                                              K &fy) {
  const K s0 = t[0] * de[0] + t[1] * de[1] + t[2] * de[2];
  const K s1 = t[3] * de[0] + t[4] * de[1] + t[5] * de[2];
  const K s2 = t[6] * de[0] + t[7] * de[1] + t[8] * de[2];
  const K gx = a == 0 ? g[0] : (a == 1 ? g[2] : -(g[0] + g[2]));
  const K gy = a == 0 ? g[1] : (a == 1 ? g[3] : -(g[1] + g[3]));
  fx = s0 * gx + s2 * gy;
  fy = s2 * gx + s1 * gy;
}

// p_new = z + beta p of a node, rebuilt from the stored (p, z).
template <typename K>
__device__ __forceinline__ typename V<K>::T2 qs_pnew(const QkParams<K> &I, int j, K beta) {
  const typename V<K>::T4 v = I.pz[j];
  typename V<K>::T2 o;
  o.x = fma(beta, v.x, v.y);
  o.y = fma(beta, v.z, v.w);
  return o;
}

// Jacobi diagonal of K_T (one unit displacement per dof through the stored
// tangents), z = r / diag, p = 0 (so that p_new = z); rho = r.z and |r_0|.
template <typename K>
__global__ void __launch_bounds__(256) k_qs_setup(QkParams<K> I) {
  typedef Acc<K> AC;
  typename AC::T vals[2] = {AC::zero(), AC::zero()};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < I.N; i += gridDim.x * blockDim.x) {
    K dx = 0, dy = 0;
    for (int k = 0; k < I.D; ++k) {
      const int en = __ldg(&I.ell[(size_t)k * I.N + i]);
      if (en < 0) continue;
      const int a = en & 3;
      int n0, n1, n2;
      K t[9], g[4];
      qrec_load(I.rec + (en >> 2), n0, n1, n2, t, g);
      const K gx = a == 0 ? g[0] : (a == 1 ? g[2] : -(g[0] + g[2]));
      const K gy = a == 0 ? g[1] : (a == 1 ? g[3] : -(g[1] + g[3]));
      const K ex[3] = {gx, K(0), K(0.5) * gy}, ey[3] = {K(0), gy, K(0.5) * gx};
      K fx, fy, hx, hy;
      qs_slot_force(t, g, a, ex, fx, fy);
      qs_slot_force(t, g, a, ey, hx, hy);
      dx = radd(dx, fx);
      dy = radd(dy, hy);
    }
    const typename V<K>::T2 r = I.r[i];
    typename V<K>::T2 dg;
    dg.x = (qs_fx(I.bc, i) || !(dx > K(0))) ? K(1) : dx;
    dg.y = (qs_fy(I.bc, i) || !(dy > K(0))) ? K(1) : dy;
    I.dg[i] = dg;
    typename V<K>::T4 pz;
    pz.x = K(0);
    pz.y = r.x / dg.x;
    pz.z = K(0);
    pz.w = r.y / dg.y;
    I.pz[i] = pz;
    vals[0] = AC::add(vals[0], AC::add(AC::prod(r.x, pz.y), AC::prod(r.y, pz.w)));
    vals[1] = AC::add(vals[1], AC::add(AC::prod(r.x, r.x), AC::prod(r.y, r.y)));
  }
  __shared__ double tot[2];
  if (reduce_last<K, 2>(vals, I.part, I.ticket, tot) && threadIdx.x == 0) {
    QsScalars &S = *I.qs;
    S.rho = tot[0];
    S.rr0 = tot[1];
    S.beta = 0.0;
    S.beta_f = 0.f;
    S.iters = 0;
    S.status = 0;
    S.done = (tot[1] == 0.0) ? 1 : 0;
  }
}

// Element pass of q = K_T p_new: per element (threads over consecutive
// records, so the record loads coalesce) the strain of p_new (rebuilt from
// (p, z) with beta at the three nodes), the stress T de and the three slot
// forces.  A no-op once the solve is done.
template <typename K>
__global__ void __launch_bounds__(256) k_qs_elem_apply(QkParams<K> I, int Ne) {
  typedef typename V<K>::T2 K2;
  if (I.qs->done) return;
  const K beta = sizeof(K) == 4 ? (K)I.qs->beta_f : (K)I.qs->beta;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < Ne; e += gridDim.x * blockDim.x) {
    int n0, n1, n2;
    K t[9], g[4];
    qrec_load(I.rec + e, n0, n1, n2, t, g);
    const K2 p0 = qs_pnew(I, n0, beta), p1 = qs_pnew(I, n1, beta), p2 = qs_pnew(I, n2, beta);
    const K ax0 = p0.x - p2.x, ax1 = p1.x - p2.x, ay0 = p0.y - p2.y, ay1 = p1.y - p2.y;
    const K de[3] = {g[0] * ax0 + g[2] * ax1, g[1] * ay0 + g[3] * ay1,
                     K(0.5) * (g[1] * ax0 + g[3] * ax1 + g[0] * ay0 + g[2] * ay1)};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      K2 f;
      qs_slot_force(t, g, a, de, f.x, f.y);
      I.fe[(size_t)3 * e + a] = f;
    }
  }
}

// Node pass: q_i = sum of its slot forces in ascending element order, 0 on
// the fixed dofs; p_new . q -> alpha.  A no-op once the solve is done.
template <typename K>
__global__ void __launch_bounds__(256) k_qs_matvec(QkParams<K> I) {
  typedef Acc<K> AC;
  typedef typename V<K>::T2 K2;
  if (I.qs->done) return;
  const K beta = sizeof(K) == 4 ? (K)I.qs->beta_f : (K)I.qs->beta;
  typename AC::T vals[1] = {AC::zero()};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < I.N; i += gridDim.x * blockDim.x) {
    K qx = 0, qy = 0;
    for (int k = 0; k < I.D; ++k) {
      const int en = __ldg(&I.ell[(size_t)k * I.N + i]);
      if (en < 0) continue;
      const K2 f = I.fe[(size_t)3 * (en >> 2) + (en & 3)];
      qx = radd(qx, f.x);
      qy = radd(qy, f.y);
    }
    if (qs_fx(I.bc, i)) qx = K(0);
    if (qs_fy(I.bc, i)) qy = K(0);
    K2 q;
    q.x = qx;
    q.y = qy;
    I.q[i] = q;
    const K2 pn = qs_pnew(I, i, beta);
    vals[0] = AC::add(vals[0], AC::add(AC::prod(pn.x, qx), AC::prod(pn.y, qy)));
  }
  __shared__ double tot[1];
  if (reduce_last<K, 1>(vals, I.part, I.ticket, tot) && threadIdx.x == 0) {
    QsScalars &S = *I.qs;
    S.pq = tot[0];
    S.alpha = tot[0] != 0.0 ? S.rho / tot[0] : 0.0;
    S.alpha_f = (float)S.alpha;
  }
}

// x += alpha p, r -= alpha q, z = r / diag, (p, z) stored; |r|^2, r.z ->
// beta and the stop test |r| <= tol |r_0|.
template <typename K>
__global__ void __launch_bounds__(256) k_qs_update(QkParams<K> I) {
  typedef Acc<K> AC;
  typedef typename V<K>::T2 K2;
  if (I.qs->done) return;
  const K beta = sizeof(K) == 4 ? (K)I.qs->beta_f : (K)I.qs->beta;
  const K alpha = sizeof(K) == 4 ? (K)I.qs->alpha_f : (K)I.qs->alpha;
  typename AC::T vals[2] = {AC::zero(), AC::zero()};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < I.N; i += gridDim.x * blockDim.x) {
    const K2 pn = qs_pnew(I, i, beta), q = I.q[i], dg = I.dg[i];
    K2 x = I.x[i], r = I.r[i];
    x.x = fma(alpha, pn.x, x.x);
    x.y = fma(alpha, pn.y, x.y);
    r.x = fma(-alpha, q.x, r.x);
    r.y = fma(-alpha, q.y, r.y);
    if (qs_fx(I.bc, i)) r.x = K(0);
    if (qs_fy(I.bc, i)) r.y = K(0);
    I.x[i] = x;
    I.r[i] = r;
    typename V<K>::T4 pz;
    pz.x = pn.x;
    pz.y = r.x / dg.x;
    pz.z = pn.y;
    pz.w = r.y / dg.y;
    I.pz[i] = pz;
    vals[0] = AC::add(vals[0], AC::add(AC::prod(r.x, r.x), AC::prod(r.y, r.y)));
    vals[1] = AC::add(vals[1], AC::add(AC::prod(r.x, pz.y), AC::prod(r.y, pz.w)));
  }
  __shared__ double tot[2];
  if (reduce_last<K, 2>(vals, I.part, I.ticket, tot) && threadIdx.x == 0) {
    QsScalars &S = *I.qs;
    S.iters += 1;
    if (!(tot[0] == tot[0]) || isinf(tot[0])) {
      S.status = kStNonfinite;
      S.done = 1;
    } else if (S.pq == 0.0 || sqrt(tot[0]) <= I.tol * sqrt(S.rr0)) {
      S.done = 1;
    } else if (S.iters >= I.max_it) {
      S.status = kStNotConverged;
      S.done = 1;
    }
    S.beta = S.rho != 0.0 ? tot[1] / S.rho : 0.0;
    S.beta_f = (float)S.beta;
    S.rho = tot[1];
  }
}

// The tangent CG of one Newton step in one cooperative launch (persistent
// CTAs): per iteration the element pass, a grid barrier, the node pass with
// a grid all-reduce of p.q, the update with a grid all-reduce of
// (|r|^2, r.z) -- the per-row arithmetic of k_qs_elem_apply, k_qs_matvec and
// k_qs_update, with every CTA taking the same decisions from bit-identical
// totals.  B holds the barrier counter and abort flag (zeroed before the
// launch); waits are bounded, and a CTA that gives up makes every CTA leave
// and the solve report kStTimeout.
constexpr int kQsPersThreads = 512;
constexpr int kQsRowGathers = 2;  // incidence slots in flight per round in k_qs_cg_rows
template <typename K>
__global__ void __launch_bounds__(kQsPersThreads, 2) k_qs_cg_persistent(QkParams<K> I, int Ne, SolveScalars *B) {
  typedef Acc<K> AC;
  typedef typename V<K>::T2 K2;
  __shared__ typename AC::T sh[kQsPersThreads / 32][2];
  __shared__ double tot[2];
  __shared__ int ok_sh, flag;
  __shared__ double rho, rr, pq, alpha_d, beta_d;
  __shared__ int iters, status;
  QsScalars *S = I.qs;
  if (S->done) return;  // the set-up found r_0 = 0
  if (threadIdx.x == 0) {
    rho = S->rho;
    rr = 0.0;
    pq = 0.0;
    alpha_d = 0.0;
    beta_d = 0.0;
    iters = 0;
    status = 0;
  }
  __syncthreads();
  const unsigned int nb = gridDim.x;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
  unsigned int nbar = 0;
  bool done = false;
  for (;;) {
    const K beta = (K)beta_d;
    // element pass: the slot forces of K_T p_new
    for (int e = tid; e < Ne; e += stride) {
      int n0, n1, n2;
      K t[9], g[4];
      qrec_load(I.rec + e, n0, n1, n2, t, g);
      const K2 p0 = qs_pnew(I, n0, beta), p1 = qs_pnew(I, n1, beta), p2 = qs_pnew(I, n2, beta);
      const K ax0 = p0.x - p2.x, ax1 = p1.x - p2.x, ay0 = p0.y - p2.y, ay1 = p1.y - p2.y;
      const K de[3] = {g[0] * ax0 + g[2] * ax1, g[1] * ay0 + g[3] * ay1,
                       K(0.5) * (g[1] * ax0 + g[3] * ax1 + g[0] * ay0 + g[2] * ay1)};
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        K2 f;
        qs_slot_force(t, g, a, de, f.x, f.y);
        I.fe[(size_t)3 * e + a] = f;
      }
    }
    typename AC::T v0[1] = {AC::zero()};
    ++nbar;
    if (!grid_sum<K, 1>(v0, I.part + (nbar & 1u) * 2u * nb, B, nbar * nb, tot, (typename AC::T(*)[1])sh, &ok_sh))
      break;
    // node pass: q = gathered slot forces, p_new . q
    typename AC::T v1[1] = {AC::zero()};
    for (int i = tid; i < I.N; i += stride) {
      K qx = 0, qy = 0;
      for (int k = 0; k < I.D; ++k) {
        const int en = __ldg(&I.ell[(size_t)k * I.N + i]);
        if (en < 0) continue;
        const K2 f = I.fe[(size_t)3 * (en >> 2) + (en & 3)];
        qx = radd(qx, f.x);
        qy = radd(qy, f.y);
      }
      if (qs_fx(I.bc, i)) qx = K(0);
      if (qs_fy(I.bc, i)) qy = K(0);
      K2 q;
      q.x = qx;
      q.y = qy;
      I.q[i] = q;
      const K2 pn = qs_pnew(I, i, beta);
      v1[0] = AC::add(v1[0], AC::add(AC::prod(pn.x, qx), AC::prod(pn.y, qy)));
    }
    ++nbar;
    if (!grid_sum<K, 1>(v1, I.part + (nbar & 1u) * 2u * nb, B, nbar * nb, tot, (typename AC::T(*)[1])sh, &ok_sh))
      break;
    if (threadIdx.x == 0) {
      pq = tot[0];
      alpha_d = pq != 0.0 ? rho / pq : 0.0;
    }
    __syncthreads();
    const K alpha = (K)alpha_d;
    // update: x += alpha p_new, r -= alpha q, z = r / diag, (p, z) stored
    typename AC::T v2[2] = {AC::zero(), AC::zero()};
    for (int i = tid; i < I.N; i += stride) {
      const K2 pn = qs_pnew(I, i, beta), q = I.q[i], dg = I.dg[i];
      K2 x = I.x[i], r = I.r[i];
      x.x = fma(alpha, pn.x, x.x);
      x.y = fma(alpha, pn.y, x.y);
      r.x = fma(-alpha, q.x, r.x);
      r.y = fma(-alpha, q.y, r.y);
      if (qs_fx(I.bc, i)) r.x = K(0);
      if (qs_fy(I.bc, i)) r.y = K(0);
      I.x[i] = x;
      I.r[i] = r;
      typename V<K>::T4 pz;
      pz.x = pn.x;
      pz.y = r.x / dg.x;
      pz.z = pn.y;
      pz.w = r.y / dg.y;
      I.pz[i] = pz;
      v2[0] = AC::add(v2[0], AC::add(AC::prod(r.x, r.x), AC::prod(r.y, r.y)));
      v2[1] = AC::add(v2[1], AC::add(AC::prod(r.x, pz.y), AC::prod(r.y, pz.w)));
    }
    ++nbar;
    if (!grid_sum<K, 2>(v2, I.part + (nbar & 1u) * 2u * nb, B, nbar * nb, tot, sh, &ok_sh)) break;
    if (threadIdx.x == 0) {
      iters += 1;
      rr = tot[0];
      flag = 0;
      if (!(tot[0] == tot[0]) || isinf(tot[0])) {
        status = kStNonfinite;
        flag = 1;
      } else if (pq == 0.0 || sqrt(tot[0]) <= I.tol * sqrt(S->rr0)) {
        flag = 1;
      } else if (iters >= I.max_it) {
        status = kStNotConverged;
        flag = 1;
      }
      beta_d = rho != 0.0 ? tot[1] / rho : 0.0;
      rho = tot[1];
    }
    __syncthreads();
    if (flag) {
      done = true;
      break;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    S->iters = iters;
    S->rr = rr;
    S->pq = pq;
    S->rho = rho;
    S->alpha = alpha_d;
    S->beta = beta_d;
    S->status = done ? status : kStTimeout;
    S->done = 1;
  }
}

// The 2 x 2 block K_ab of the element tangent (the force on slot a per unit
// displacement of slot b): columns are the unit x and y displacements.
template <typename K>
__device__ __forceinline__ float4 qs_block(const K (&t)[9], const K (&g)[4], int a, int b) {
  const K gx = b == 0 ? g[0] : (b == 1 ? g[2] : -(g[0] + g[2]));
  const K gy = b == 0 ? g[1] : (b == 1 ? g[3] : -(g[1] + g[3]));
  const K ex[3] = {gx, K(0), K(0.5) * gy}, ey[3] = {K(0), gy, K(0.5) * gx};
  K xx, yx, xy, yy;
  qs_slot_force(t, g, a, ex, xx, yx);
  qs_slot_force(t, g, a, ey, xy, yy);
  return make_float4((float)xx, (float)xy, (float)yx, (float)yy);
}

// The pair block K_ab evaluated the same way from either end (the lower
// slot's block, transposed for the higher), so that the stored operator is
// exactly symmetric, as CG needs.
template <typename K>
__device__ __forceinline__ float4 qs_pair_block(const K (&t)[9], const K (&g)[4], int a, int b) {
  if (a < b) return qs_block(t, g, a, b);
  const float4 m = qs_block(t, g, b, a);
  return make_float4(m.x, m.z, m.y, m.w);
}

// Entry records of the tangent, once per Newton step (node-parallel over
// the incidence): per slot the neighbour offsets and blocks K_ab, K_ac;
// empty slots get zero offsets and zero blocks (they add an exact 0).
__global__ void __launch_bounds__(256) k_qs_entry_build(QkParams<float> I) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < I.N; i += gridDim.x * blockDim.x) {
    float4 acc[6];
    uint2 map = make_uint2(0xffffffffu, 0xffffffffu);
    if (I.nbk) {
#pragma unroll
      for (int j = 0; j < 6; ++j) acc[j] = make_float4(0.f, 0.f, 0.f, 0.f);
      map = __ldg(&I.nmap[i]);
    }
    const uint32_t fm = I.fmap ? __ldg(&I.fmap[i]) : 0u;
    for (int k = 0; k < I.D; ++k) {
      const size_t q = (size_t)k * I.N + i;
      const int en = __ldg(&I.ell[q]);
      if (en < 0) {
        if (!I.nbk) {
          I.ofs[q] = 0u;
          I.kb[q] = make_float4(0.f, 0.f, 0.f, 0.f);
          I.kc[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        continue;
      }
      const int a = en & 3;
      int n0, n1, n2;
      float t[9], g[4];
      qrec_load(I.rec + (en >> 2), n0, n1, n2, t, g);
      const int b = a == 0 ? 1 : 0, c = a == 2 ? 1 : 2;
      const float4 kb = qs_pair_block(t, g, a, b), kc = qs_pair_block(t, g, a, c);
      if (I.nbk) {
        // merged: each block into its neighbour's slot, in slot order
        const unsigned m = ((k < 4 ? map.x : map.y) >> (8 * (k & 3))) & 0xffu;
        const unsigned jb = m & 15u, jc = m >> 4;
#pragma unroll
        for (int j = 0; j < 6; ++j) {
          if (jb == (unsigned)j) {
            acc[j].x = __fadd_rn(acc[j].x, kb.x);
            acc[j].y = __fadd_rn(acc[j].y, kb.y);
            acc[j].z = __fadd_rn(acc[j].z, kb.z);
            acc[j].w = __fadd_rn(acc[j].w, kb.w);
          }
          if (jc == (unsigned)j) {
            acc[j].x = __fadd_rn(acc[j].x, kc.x);
            acc[j].y = __fadd_rn(acc[j].y, kc.y);
            acc[j].z = __fadd_rn(acc[j].z, kc.z);
            acc[j].w = __fadd_rn(acc[j].w, kc.w);
          }
        }
        continue;
      }
      if (I.fmap) {
        // fan position; (K_ab, K_ac) ordered counter-clockwise from the
        // vertex, which (b, c) is for slots 0 and 2 and reverses for slot 1
        const size_t qf = (size_t)((fm >> (4 * k)) & 15u) * I.N + i;
        I.kb[qf] = a == 1 ? kc : kb;
        I.kc[qf] = a == 1 ? kb : kc;
        continue;
      }
      const int nb = b == 0 ? n0 : n1, nc = c == 1 ? n1 : n2;
      I.ofs[q] = (uint32_t)(uint16_t)(int16_t)(nb - i) | ((uint32_t)(uint16_t)(int16_t)(nc - i) << 16);
      I.kb[q] = kb;
      I.kc[q] = kc;
    }
    if (I.nbk) {
#pragma unroll
      for (int j = 0; j < 6; ++j) I.nbk[(size_t)j * I.N + i] = acc[j];
    }
  }
}

// The tangent CG of one Newton step on the entry records, one cooperative
// launch: per iteration the node rows q_i = sum_k (K_ab (p_b - p_i) +
// K_ac (p_c - p_i)) with a grid all-reduce of p.q, then the update with a grid
// all-reduce of (|r|^2, r.z) -- two grid barriers per iteration instead of
// the element pass's three.  Decisions and bounded waits as in
// k_qs_cg_persistent; the totals and the scalar step (alpha, beta, the stop
// test |r|^2 <= tol^2 |r_0|^2) in double-word FP32, as in the damage
// solve's single-reduction loops (no FP64 instruction in the loop).
template <int U>
__global__ void __launch_bounds__(kQsPersThreads, 2) k_qs_cg_rows(QkParams<float> I, SolveScalars *B) {
  typedef Acc<float> AC;
  typedef float2 K2;
  __shared__ typename AC::T sh[kQsPersThreads / 32][2];
  __shared__ DF tot[2];
  __shared__ int ok_sh, flag;
  __shared__ DF rho, rr, pq, alpha_d, beta_d, thr2;
  __shared__ int iters, status;
  QsScalars *S = I.qs;
  if (S->done) return;
  if (threadIdx.x == 0) {
    rho = df_from(S->rho);
    rr = DF{0.f, 0.f};
    pq = DF{0.f, 0.f};
    alpha_d = DF{0.f, 0.f};
    beta_d = DF{0.f, 0.f};
    thr2 = df_from(I.tol * I.tol * S->rr0);
    iters = 0;
    status = 0;
  }
  __syncthreads();
  const unsigned int nb = gridDim.x;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
  unsigned int nbar = 0;
  bool done = false;
  // rows last first on odd iterations: each pass starts on the blocks and
  // vectors the previous one touched last (the working set exceeds L2)
  const int ilast = tid < I.N ? tid + (I.N - 1 - tid) / stride * stride : tid - stride;
  for (;;) {
    const float beta = beta_d.hi;
    const bool rev = (iters & 1) != 0;
    const int istep = rev ? -stride : stride;
    // rows: q = K_T p_new on the free dofs, p_new . q
    typename AC::T v1[1] = {AC::zero()};
    for (int i = rev ? ilast : tid; rev ? i >= tid : i < I.N; i += istep) {
      const K2 pc = qs_pnew(I, i, beta);
      float qx = 0.f, qy = 0.f;
      if (I.nbk) {
        // merged row: all six records, then the six neighbour gathers in
        // flight, then sum_j K_ij (p_j - p_i) in slot order (padding slots
        // have offset 0 and add an exact 0)
        uint32_t w[3];
        float4 kk[6];
#pragma unroll
        for (int j = 0; j < 3; ++j) w[j] = __ldg(&I.nbo[(size_t)j * I.N + i]);
#pragma unroll
        for (int j = 0; j < 6; ++j) kk[j] = __ldg(&I.nbk[(size_t)j * I.N + i]);
        K2 pj[6];
#pragma unroll
        for (int j = 0; j < 6; ++j) {
          const uint32_t x = w[j >> 1];
          pj[j] = qs_pnew(I, i + ((j & 1) ? (int)x >> 16 : (int)(int16_t)(x & 0xffffu)), beta);
        }
#pragma unroll
        for (int j = 0; j < 6; ++j) {
          const float dx = pj[j].x - pc.x, dy = pj[j].y - pc.y;
          qx = __fadd_rn(qx, fmaf(kk[j].x, dx, __fmul_rn(kk[j].y, dy)));
          qy = __fadd_rn(qy, fmaf(kk[j].z, dx, __fmul_rn(kk[j].w, dy)));
        }
      }
      if (!I.nbk && I.fno) {
        // fan order: the six distinct neighbours gathered once, then per
        // fan position K_b (p_{v_k} - p_i) + K_c (p_{v_{k+1}} - p_i) in
        // position order (positions past the fan hold zero blocks)
        uint32_t w[3];
        float4 bb[6], cc[6];
#pragma unroll
        for (int j = 0; j < 3; ++j) w[j] = __ldg(&I.fno[(size_t)j * I.N + i]);
        const int m = (int)(__ldg(&I.fmap[i]) >> 24);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          const bool in = k < I.D;
          bb[k] = in ? __ldg(&I.kb[(size_t)k * I.N + i]) : make_float4(0.f, 0.f, 0.f, 0.f);
          cc[k] = in ? __ldg(&I.kc[(size_t)k * I.N + i]) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        K2 pv[6];
#pragma unroll
        for (int j = 0; j < 6; ++j) {
          const uint32_t x = w[j >> 1];
          pv[j] = qs_pnew(I, i + ((j & 1) ? (int)x >> 16 : (int)(int16_t)(x & 0xffffu)), beta);
        }
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          const K2 pb = pv[k], pcc = (k + 1 == m) ? pv[0] : pv[k < 5 ? k + 1 : 0];
          const float bx = pb.x - pc.x, by = pb.y - pc.y, cx = pcc.x - pc.x, cy = pcc.y - pc.y;
          const float fx = fmaf(bb[k].x, bx, fmaf(bb[k].y, by, fmaf(cc[k].x, cx, __fmul_rn(cc[k].y, cy))));
          const float fy = fmaf(bb[k].z, bx, fmaf(bb[k].w, by, fmaf(cc[k].z, cx, __fmul_rn(cc[k].w, cy))));
          qx = __fadd_rn(qx, fx);
          qy = __fadd_rn(qy, fy);
        }
      }
      for (int k = 0; k < I.D && !I.nbk && !I.fno; k += U) {
        uint32_t w[U];
        float4 bb[U], cc[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const bool in = k + u < I.D;
          const size_t q = (size_t)(k + u) * I.N + i;
          w[u] = in ? __ldg(&I.ofs[q]) : 0u;
          bb[u] = in ? __ldg(&I.kb[q]) : make_float4(0.f, 0.f, 0.f, 0.f);
          cc[u] = in ? __ldg(&I.kc[q]) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const K2 pb = qs_pnew(I, i + (int)(int16_t)(w[u] & 0xffffu), beta);
          const K2 pcc = qs_pnew(I, i + ((int)w[u] >> 16), beta);
          const float bx = pb.x - pc.x, by = pb.y - pc.y, cx = pcc.x - pc.x, cy = pcc.y - pc.y;
          const float fx = fmaf(bb[u].x, bx, fmaf(bb[u].y, by, fmaf(cc[u].x, cx, __fmul_rn(cc[u].y, cy))));
          const float fy = fmaf(bb[u].z, bx, fmaf(bb[u].w, by, fmaf(cc[u].z, cx, __fmul_rn(cc[u].w, cy))));
          qx = __fadd_rn(qx, fx);
          qy = __fadd_rn(qy, fy);
        }
      }
      if (qs_fx(I.bc, i)) qx = 0.f;
      if (qs_fy(I.bc, i)) qy = 0.f;
      I.q[i] = make_float2(qx, qy);
      v1[0] = AC::add(v1[0], AC::add(AC::prod(pc.x, qx), AC::prod(pc.y, qy)));
    }
    ++nbar;
    if (!grid_sum<float, 1>(v1, I.part + (nbar & 1u) * 2u * nb, B, nbar * nb, tot, (typename AC::T(*)[1])sh,
                            &ok_sh))
      break;
    if (threadIdx.x == 0) {
      pq = tot[0];
      alpha_d = pq.hi != 0.f ? df_div(rho, pq) : DF{0.f, 0.f};
    }
    __syncthreads();
    const float alpha = alpha_d.hi;
    typename AC::T v2[2] = {AC::zero(), AC::zero()};
    for (int i = rev ? ilast : tid; rev ? i >= tid : i < I.N; i += istep) {
      const K2 pn = qs_pnew(I, i, beta), q = I.q[i], dg = I.dg[i];
      K2 x = I.x[i], r = I.r[i];
      x.x = fmaf(alpha, pn.x, x.x);
      x.y = fmaf(alpha, pn.y, x.y);
      r.x = fmaf(-alpha, q.x, r.x);
      r.y = fmaf(-alpha, q.y, r.y);
      if (qs_fx(I.bc, i)) r.x = 0.f;
      if (qs_fy(I.bc, i)) r.y = 0.f;
      I.x[i] = x;
      I.r[i] = r;
      const float4 pz = make_float4(pn.x, r.x / dg.x, pn.y, r.y / dg.y);
      I.pz[i] = pz;
      v2[0] = AC::add(v2[0], AC::add(AC::prod(r.x, r.x), AC::prod(r.y, r.y)));
      v2[1] = AC::add(v2[1], AC::add(AC::prod(r.x, pz.y), AC::prod(r.y, pz.w)));
    }
    ++nbar;
    if (!grid_sum<float, 2>(v2, I.part + (nbar & 1u) * 2u * nb, B, nbar * nb, tot, sh, &ok_sh)) break;
    if (threadIdx.x == 0) {
      iters += 1;
      rr = tot[0];
      flag = 0;
      if (!df_finite(tot[0])) {
        status = kStNonfinite;
        flag = 1;
      } else if (pq.hi == 0.f || df_le(tot[0], thr2)) {
        flag = 1;
      } else if (iters >= I.max_it) {
        status = kStNotConverged;
        flag = 1;
      }
      beta_d = rho.hi != 0.f ? df_div(tot[1], rho) : DF{0.f, 0.f};
      rho = tot[1];
    }
    __syncthreads();
    if (flag) {
      done = true;
      break;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    S->iters = iters;
    S->rr = df_to(rr);
    S->pq = df_to(pq);
    S->rho = df_to(rho);
    S->alpha = df_to(alpha_d);
    S->beta = df_to(beta_d);
    S->status = done ? status : kStTimeout;
    S->done = 1;
  }
}

// ------------------------------------------- resident tangent CG (fan rows)
//
// k_qs_cg_rows on fan-order rows with CTA b owning the rows [b R, (b+1) R)
// for the whole solve (R rows, a multiple of 4): per row x, r, (p, z), q,
// the Jacobi diagonal, the fan words and the fan length with the row's
// boundary flags stay in shared memory (kQsResWords words a row), so a
// pass reads from global memory only the rows' pair blocks and the (p, z)
// of neighbours another CTA owns, and the update pass works in shared
// memory alone; a row writes its (p, z) to global memory only if it lies
// within H (the mesh's element span, which bounds every neighbour offset)
// of either end of the range, where another CTA may read it.  Per row the
// arithmetic of k_qs_cg_rows' fan branch and update; the dot products'
// partial sums are grouped by CTA range.  x goes back to global memory at
// the end.  Layout (words): x [0, 2R), r [2R, 4R), (p, z) [4R, 8R), q
// [8R, 10R), diagonal [10R, 12R), fan words [12R, 15R), fan length | bc
// << 8 [15R, 16R).
constexpr int kQsResThreads = 1024;
constexpr int kQsResWords = 16;

__device__ __forceinline__ float2 qs_pnew_v(const float4 v, float beta) {
  return make_float2(fmaf(beta, v.x, v.y), fmaf(beta, v.z, v.w));
}

// Row l's q = K_T p_new (fan branch of k_qs_cg_rows) and its p_new . q.
__device__ __forceinline__ void qs_res_row(const QkParams<float> &I, int row0, int nr, int R, uint32_t *rs,
                                           int l, float beta, DF &v1) {
  typedef Acc<float> AC;
  const float4 *pzs = reinterpret_cast<const float4 *>(rs + 4 * R);
  float2 *qsm = reinterpret_cast<float2 *>(rs + 8 * R);
  const int i = row0 + l;
  const uint32_t mt = rs[15 * R + l];
  const float2 pc = qs_pnew_v(pzs[l], beta);
  const uint32_t w[3] = {rs[12 * R + l], rs[13 * R + l], rs[14 * R + l]};
  const int m = (int)(mt & 0xffu);
  float4 bb[6], cc[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const bool in = k < I.D;
    bb[k] = in ? __ldg(&I.kb[(size_t)k * I.N + i]) : make_float4(0.f, 0.f, 0.f, 0.f);
    cc[k] = in ? __ldg(&I.kc[(size_t)k * I.N + i]) : make_float4(0.f, 0.f, 0.f, 0.f);
  }
  float2 pv[6];
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    const int ln = l + fan_offset(w, j);
    pv[j] = qs_pnew_v((unsigned)ln < (unsigned)nr ? pzs[ln] : I.pz[row0 + ln], beta);
  }
  float qx = 0.f, qy = 0.f;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const float2 pb = pv[k], pcc = (k + 1 == m) ? pv[0] : pv[k < 5 ? k + 1 : 0];
    const float bx = pb.x - pc.x, by = pb.y - pc.y, cx = pcc.x - pc.x, cy = pcc.y - pc.y;
    const float fx = fmaf(bb[k].x, bx, fmaf(bb[k].y, by, fmaf(cc[k].x, cx, __fmul_rn(cc[k].y, cy))));
    const float fy = fmaf(bb[k].z, bx, fmaf(bb[k].w, by, fmaf(cc[k].z, cx, __fmul_rn(cc[k].w, cy))));
    qx = __fadd_rn(qx, fx);
    qy = __fadd_rn(qy, fy);
  }
  const uint32_t bcf = mt >> 8;
  if (bcf & kQsFixX) qx = 0.f;
  if (bcf & (kQsFixY | kQsLoaded)) qy = 0.f;
  qsm[l] = make_float2(qx, qy);
  v1 = AC::add(v1, AC::add(AC::prod(pc.x, qx), AC::prod(pc.y, qy)));
}

// Row l's update (k_qs_cg_rows' second phase) in shared memory; |r|^2 and
// r.z.
__device__ __forceinline__ void qs_res_update(const QkParams<float> &I, int row0, int nr, int R, int H,
                                              uint32_t *rs, int l, float alpha, float beta, DF (&v2)[2]) {
  typedef Acc<float> AC;
  float2 *xs = reinterpret_cast<float2 *>(rs);
  float2 *rsv = reinterpret_cast<float2 *>(rs + 2 * R);
  float4 *pzs = reinterpret_cast<float4 *>(rs + 4 * R);
  const float2 *qsm = reinterpret_cast<const float2 *>(rs + 8 * R);
  const float2 *dgs = reinterpret_cast<const float2 *>(rs + 10 * R);
  const uint32_t bcf = rs[15 * R + l] >> 8;
  const float2 pn = qs_pnew_v(pzs[l], beta), q = qsm[l], dg = dgs[l];
  float2 x = xs[l], r = rsv[l];
  x.x = fmaf(alpha, pn.x, x.x);
  x.y = fmaf(alpha, pn.y, x.y);
  r.x = fmaf(-alpha, q.x, r.x);
  r.y = fmaf(-alpha, q.y, r.y);
  if (bcf & kQsFixX) r.x = 0.f;
  if (bcf & (kQsFixY | kQsLoaded)) r.y = 0.f;
  xs[l] = x;
  rsv[l] = r;
  const float4 pz = make_float4(pn.x, r.x / dg.x, pn.y, r.y / dg.y);
  pzs[l] = pz;
  if (l < H || l >= nr - H) I.pz[row0 + l] = pz;  // another CTA's neighbour
  v2[0] = AC::add(v2[0], AC::add(AC::prod(r.x, r.x), AC::prod(r.y, r.y)));
  v2[1] = AC::add(v2[1], AC::add(AC::prod(r.x, pz.y), AC::prod(r.y, pz.w)));
}

__global__ void __launch_bounds__(kQsResThreads, 1) k_qs_cg_res(QkParams<float> I, SolveScalars *B, int R, int H) {
  typedef Acc<float> AC;
  __shared__ typename AC::T sh[kQsResThreads / 32][2];
  __shared__ DF tot[2];
  __shared__ int ok_sh, flag;
  __shared__ DF rho, rr, pq, alpha_d, beta_d, thr2;
  __shared__ int iters, status;
  extern __shared__ __align__(16) uint32_t qres_smem[];
  uint32_t *rs = qres_smem;
  QsScalars *S = I.qs;
  if (S->done) return;
  const int row0 = (int)blockIdx.x * R;
  const int nr = max(0, min(R, I.N - row0));
  for (int l = threadIdx.x; l < nr; l += blockDim.x) {
    const int i = row0 + l;
    reinterpret_cast<float2 *>(rs)[l] = I.x[i];
    reinterpret_cast<float2 *>(rs + 2 * R)[l] = I.r[i];
    reinterpret_cast<float4 *>(rs + 4 * R)[l] = I.pz[i];
    reinterpret_cast<float2 *>(rs + 10 * R)[l] = I.dg[i];
#pragma unroll
    for (int k = 0; k < 3; ++k) rs[(12 + k) * R + l] = __ldg(&I.fno[(size_t)k * I.N + i]);
    rs[15 * R + l] = (__ldg(&I.fmap[i]) >> 24) | ((uint32_t)I.bc[i] << 8);
  }
  if (threadIdx.x == 0) {
    rho = df_from(S->rho);
    rr = DF{0.f, 0.f};
    pq = DF{0.f, 0.f};
    alpha_d = DF{0.f, 0.f};
    beta_d = DF{0.f, 0.f};
    thr2 = df_from(I.tol * I.tol * S->rr0);
    iters = 0;
    status = 0;
  }
  __syncthreads();
  const unsigned int nb = gridDim.x;
  const int T = (int)blockDim.x, t = (int)threadIdx.x;
  const int llast = t < nr ? t + (nr - 1 - t) / T * T : t - T;
  unsigned int nbar = 0;
  bool done = false;
  for (;;) {
    const float beta = beta_d.hi;
    const bool rev = (iters & 1) != 0;  // rows last first on odd iterations
    const int lstep = rev ? -T : T;
    typename AC::T v1[1] = {AC::zero()};
    for (int l = rev ? llast : t; rev ? l >= t : l < nr; l += lstep) qs_res_row(I, row0, nr, R, rs, l, beta, v1[0]);
    ++nbar;
    if (!grid_sum<float, 1>(v1, I.part + (nbar & 1u) * 2u * nb, B, nbar * nb, tot, (typename AC::T(*)[1])sh,
                            &ok_sh))
      break;
    if (threadIdx.x == 0) {
      pq = tot[0];
      alpha_d = pq.hi != 0.f ? df_div(rho, pq) : DF{0.f, 0.f};
    }
    __syncthreads();
    const float alpha = alpha_d.hi;
    typename AC::T v2[2] = {AC::zero(), AC::zero()};
    for (int l = rev ? llast : t; rev ? l >= t : l < nr; l += lstep)
      qs_res_update(I, row0, nr, R, H, rs, l, alpha, beta, v2);
    ++nbar;
    if (!grid_sum<float, 2>(v2, I.part + (nbar & 1u) * 2u * nb, B, nbar * nb, tot, sh, &ok_sh)) break;
    if (threadIdx.x == 0) {
      iters += 1;
      rr = tot[0];
      flag = 0;
      if (!df_finite(tot[0])) {
        status = kStNonfinite;
        flag = 1;
      } else if (pq.hi == 0.f || df_le(tot[0], thr2)) {
        flag = 1;
      } else if (iters >= I.max_it) {
        status = kStNotConverged;
        flag = 1;
      }
      beta_d = rho.hi != 0.f ? df_div(tot[1], rho) : DF{0.f, 0.f};
      rho = tot[1];
    }
    __syncthreads();
    if (flag) {
      done = true;
      break;
    }
  }
  for (int l = threadIdx.x; l < nr; l += blockDim.x) I.x[row0 + l] = reinterpret_cast<const float2 *>(rs)[l];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    S->iters = iters;
    S->rr = df_to(rr);
    S->pq = df_to(pq);
    S->rho = df_to(rho);
    S->alpha = df_to(alpha_d);
    S->beta = df_to(beta_d);
    S->status = done ? status : kStTimeout;
    S->done = 1;
  }
}

// u += x on the free dofs.
template <typename R, typename K>
__global__ void __launch_bounds__(256) k_qs_apply(QsParams<R, K> Q) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Q.P.N; i += gridDim.x * blockDim.x) {
    typename Params<R>::R2 u = Q.P.u[i];
    const typename V<K>::T2 x = Q.I.x[i];
    if (!qs_fx(Q.I.bc, i)) u.x += (R)x.x;
    if (!qs_fy(Q.I.bc, i)) u.y += (R)x.y;
    Q.P.u[i] = u;
  }
}

// History H = max(H, psi+(u)) per element (the owner-entry rule of the
// dynamic step, element by element).
template <typename R>
__global__ void __launch_bounds__(256) k_qs_history(Params<R> P) {
  typedef typename Params<R>::R4 R4;
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
