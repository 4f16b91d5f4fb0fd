// batch.cuh -- many independent plates in one launch per kernel (sm_103a).
//
// The plates are concatenated into one mesh whose node ranges start on
// multiples of 256 (padding nodes have no elements, no mass and are fixed),
// so every 256-node block belongs to one plate.  Each plate keeps its own
// time step, fracture toughness and regularisation length, traction-ramp
// table, CG scalars and convergence: reductions are per plate (the plate's
// last block sums its blocks' partials) and a converged plate's blocks skip
// the CG kernels while the others iterate.  The step is the same staggered
// step as for one plate (Sec. 2.2); the same entry functions are used.
#pragma once
#include "kernels.cuh"

namespace pff {

constexpr int kThreadsBatch = 256;  // nodes per node block (plates start on block boundaries)

// Per-plate coefficients (device array, one per plate).
struct PlateC {
  double dt;        // the plate's stable step
  double tol;       // relative CG tolerance
  float kappa, cbase, wbase, rscale;  // damage coefficients (FP32 path)
  double kappa_d, cbase_d, wbase_d, rscale_d;
  int32_t blk0, nblk;  // first node block and number of node blocks
  int32_t cta0, ncta;  // the plate's CTA group in the persistent CG launch
};

struct Batch {
  int32_t nplates;
  int32_t nsteps1;            // stride of the S table (steps of the run + 1)
  const int32_t *blk_plate;   // node block -> plate
  const PlateC *pc;
  const double *Stab;         // nplates x nsteps1 traction scales
  SolveScalars *sc;           // nplates
  unsigned int *tick;         // nplates block tickets (reductions)
  unsigned int *gtick;        // plate ticket for the global loop decision
  int32_t *nactive;           // plates still iterating
  int32_t *iters_log;         // device, nsteps x nplates (nullable)
  const int2 *cta_plate;      // persistent CG: CTA -> (plate, rank in the plate's group)
};

template <typename R>
__device__ __forceinline__ void plate_apply(Params<R> &Q, const Batch &B, int p) {
  const PlateC &c = B.pc[p];
  Q.dt = c.dt;
  Q.tol = c.tol;
  if (sizeof(R) == 4) {
    Q.kappa = (R)c.kappa;
    Q.cbase = (R)c.cbase;
    Q.wbase = (R)c.wbase;
    Q.rscale = (R)c.rscale;
  } else {
    Q.kappa = (R)c.kappa_d;
    Q.cbase = (R)c.cbase_d;
    Q.wbase = (R)c.wbase_d;
    Q.rscale = (R)c.rscale_d;
  }
  Q.sc = B.sc + p;
  Q.Stab = B.Stab + (size_t)p * B.nsteps1;
}

// Per-plate version of reduce_last: the plate's blocks are
// [blk0, blk0 + nblk); the last of them to finish gets the totals.
template <typename R, int NV>
__device__ __forceinline__ bool reduce_plate(typename Acc<R>::T (&v)[NV], double *part, unsigned int *ticket,
                                             int blk0, int nblk, double *tot) {
  typedef Acc<R> A;
  typedef typename A::T T;
  __shared__ T sh[32][NV];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    T s = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s = A::add(s, A::shfl(s, o));
    if (lane == 0) sh[wid][k] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 0; k < NV; ++k) {
      T s = sh[0][k];
      for (int w = 1; w < nw; ++w) s = A::add(s, sh[w][k]);
      A::store(&part[(size_t)blockIdx.x * NV + k], s);
    }
    __threadfence();
    const unsigned int t = atomicAdd(ticket, 1u);
    last = (t == (unsigned)nblk - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  T acc[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    acc[k] = A::zero();
    for (int j0 = threadIdx.x; j0 < nblk; j0 += 8 * blockDim.x) {
      T buf[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int j = j0 + u * blockDim.x;
        buf[u] = j < nblk ? A::load(&part[(size_t)(blk0 + j) * NV + k]) : A::zero();
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) acc[k] = A::add(acc[k], buf[u]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    T s = acc[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s = A::add(s, A::shfl(s, o));
    if (lane == 0) sh[wid][k] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 0; k < NV; ++k) {
      T s = sh[0][k];
      for (int w = 1; w < nw; ++w) s = A::add(s, sh[w][k]);
      tot[k] = A::to_d(s);
    }
    *ticket = 0u;
  }
  __syncthreads();
  return true;
}

// The last plate to report sets the loop condition: continue while any
// plate is still iterating.  Called by one thread of a plate's last block.
template <typename R>
__device__ __forceinline__ void plate_report(const Params<R> &P, const Batch &B, bool reset_active) {
  __threadfence();
  const int expected = reset_active ? B.nplates : *B.nactive;
  const unsigned int t = atomicAdd(B.gtick, 1u);
  if (t == (unsigned)expected - 1) {
    __threadfence();
    int act = 0;
    for (int q = 0; q < B.nplates; ++q) act += __ldcg(&B.sc[q].inner_done) ? 0 : 1;
    *B.nactive = act;
    *B.gtick = 0u;
    if (P.use_cond) cudaGraphSetConditional(P.cond_inner, act > 0 ? 1u : 0u);
  }
}

// ---------------------------------------------------------------- kernels
// Launched with exactly one block per 256-node block (no grid stride).

template <typename R>
__global__ void __launch_bounds__(256) kb_predict(Params<R> P, Batch B) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P.N) return;
  const R dt = (R)B.pc[B.blk_plate[blockIdx.x]].dt, h = R(0.5) * dt * dt;
  typename Params<R>::R2 u = P.u[i], v = P.v[i], a = P.a[i];
  u.x += dt * v.x + h * a.x;
  u.y += dt * v.y + h * a.y;
  P.u[i] = u;
}

template <typename R, int U>
__global__ void __launch_bounds__(256) kb_force(Params<R> P, Batch B) {
  const int p = B.blk_plate[blockIdx.x];
  Params<R> Q = P;
  plate_apply(Q, B, p);
  const double S = Q.Stab[*P.step_ctr + 1];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P.N) return;
  R fx = 0, fy = 0;
  for (int k = 0; k < P.D; k += U) {
    int en[U];
    R cx[U], cy[U], pp[U];
#pragma unroll
    for (int u = 0; u < U; ++u) en[u] = k + u < P.D ? __ldg(&P.ell[(size_t)(k + u) * P.N + i]) : -1;
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (en[u] >= 0) force_entry(Q, en[u], cx[u], cy[u], pp[u]);
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (en[u] >= 0) {
        fx = radd(fx, cx[u]);
        fy = radd(fy, cy[u]);
        history_update(Q, en[u], pp[u]);
      }
  }
  corrector(Q, i, fx, fy, S);
}

template <typename R, int U>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 4 : 1) kb_rhs(Params<R> P, Batch B) {
  typedef typename Params<R>::R4 R4;
  typedef Acc<R> AC;
  const int p = B.blk_plate[blockIdx.x];
  Params<R> Q = P;
  plate_apply(Q, B, p);
  typename AC::T vals[3] = {AC::zero(), AC::zero(), AC::zero()};
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < P.N) {
    if (P.flags[i] & kNotch) {
      rhs_notch_node(Q, i);
      drec_notch_node(Q, i);
    } else {
      R bi = 0, dg = 0, ax = 0, a1 = 0;
      const bool merge = nb_merging(Q);
      NbAcc<R> nacc;
      nacc.zero();
      if (merge) nacc.load_map(Q, i);
      const uint32_t fm = fan_word(Q, i);
      for (int k = 0; k < P.D; k += U) {
        R4 o[U];
        typename Params<R>::R2 cf[U];
        int en[U];
#pragma unroll
        for (int u = 0; u < U; ++u) en[u] = k + u < P.D ? __ldg(&P.ell[(size_t)(k + u) * P.N + i]) : -1;
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (en[u] >= 0) o[u] = rhs_entry(Q, en[u], k + u, i, -1, merge ? &cf[u] : nullptr, fm);
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (en[u] >= 0) {
            bi = radd(bi, o[u].x);
            dg = radd(dg, o[u].y);
            ax = radd(ax, o[u].z);
            a1 = radd(a1, o[u].w);
            if (merge) nacc.add(k + u, cf[u]);
          }
      }
      rhs_node(Q, i, bi, dg, ax, a1, vals);
      if (merge) nacc.store(Q, i);
    }
  }
  __shared__ double tot[3];
  const PlateC &c = B.pc[p];
  if (reduce_plate<R, 3>(vals, P.part, B.tick + p, c.blk0, c.nblk, tot) && threadIdx.x == 0) {
    Params<R> F = Q;
    F.use_cond = 0;  // the global decision is taken in plate_report
    rhs_finish(F, tot);
    Q.sc->inner_done = Q.sc->done;
    plate_report(P, B, true);
  }
}

// FP32: at most 40 registers (six blocks per SM; the gather is latency-bound).
template <typename R, int U>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 6 : 1) kb_matvec(Params<R> P, Batch B) {
  typedef Acc<R> AC;
  const int p = B.blk_plate[blockIdx.x];
  if (B.sc[p].inner_done) return;  // converged plate
  Params<R> Q = P;
  plate_apply(Q, B, p);
  typename AC::T vals[1] = {AC::zero()};
  const R beta = sc_beta<R>(Q.sc);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < P.N) {
    R q = 0;
    if (!is_fixed(Q, i)) {
      const R pc = pnew(Q, i, beta);
      bool done = false;
      if constexpr (sizeof(R) == 4) {
        if (has_erec(Q)) {
          // FP32 entry records or merged rows (see matvec_rows)
          q = erec_row<U>(Q, i, beta, pc);
          done = true;
        }
      } else if (Q.nbc) {  // FP64 merged rows
        q = nb_row_any(Q, i, Q.diag[i] * pc, [&](int j) { return pnew(Q, j, beta); });
        done = true;
      } else if (Q.ecfd) {  // FP64 entry records
        q = erec_row_d<U>(Q, i, beta, pc);
        done = true;
      }
      for (int k = 0; k < P.D && !done; k += U) {
        R c[U];
        int en[U];
#pragma unroll
        for (int u = 0; u < U; ++u) en[u] = k + u < P.D ? __ldg(&P.ell[(size_t)(k + u) * P.N + i]) : -1;
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (en[u] >= 0) c[u] = mv_entry(Q, en[u], beta, pc);
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (en[u] >= 0) q = radd(q, c[u]);
      }
      vals[0] = AC::add(vals[0], AC::prod(pc, Q.rscale * q));
    }
    P.q[i] = q;
  }
  __shared__ double tot[1];
  const PlateC &c = B.pc[p];
  if (reduce_plate<R, 1>(vals, P.part, B.tick + p, c.blk0, c.nblk, tot) && threadIdx.x == 0) matvec_finish(Q, tot);
}

constexpr int kbUpdatePairThreads = 128;  // FP32 kb_update: 128 threads x 2 rows = one 256-row block

template <typename R>
__global__ void __launch_bounds__(256) kb_update(Params<R> P, Batch B) {
  typedef typename Params<R>::R2 R2;
  typedef Acc<R> AC;
  const int p = B.blk_plate[blockIdx.x];
  if (B.sc[p].inner_done) return;
  Params<R> Q = P;
  plate_apply(Q, B, p);
  typename AC::T vals[3] = {AC::zero(), AC::zero(), AC::zero()};
  const R beta = sc_beta<R>(Q.sc), alpha = sc_alpha<R>(Q.sc);
  bool proj = false;
  if constexpr (sizeof(R) == 4) {
    // FP32: a block of kbUpdatePairThreads threads updates its 256 rows in
    // pairs with vector loads and stores (the padded batch length is a
    // multiple of 256, so every pair lies inside one plate's block)
    const int j = blockIdx.x * blockDim.x + threadIdx.x, i = 2 * j;
    if (i < P.N) {
      const uchar2 f = reinterpret_cast<const uchar2 *>(P.flags)[j];
      float2 xv = reinterpret_cast<const float2 *>(P.x)[j], rv = reinterpret_cast<const float2 *>(P.r)[j];
      const float2 qv = reinterpret_cast<const float2 *>(P.q)[j], dv = reinterpret_cast<const float2 *>(P.dinv)[j];
      const float4 pv = reinterpret_cast<const float4 *>(P.pz)[j];
      R2 pz0, pz1;
      pz0.x = pv.x; pz0.y = pv.y;
      pz1.x = pv.z; pz1.y = pv.w;
      const bool fix0 = (f.x & kNotch) || (Q.freef && !Q.freef[i]);
      const bool fix1 = (f.y & kNotch) || (Q.freef && !Q.freef[i + 1]);
      if (!fix0) update_node(Q, i, alpha, beta, xv.x, rv.x, pz0, qv.x, dv.x, vals, proj);
      if (!fix1) update_node(Q, i + 1, alpha, beta, xv.y, rv.y, pz1, qv.y, dv.y, vals, proj);
      reinterpret_cast<float2 *>(P.x)[j] = xv;
      reinterpret_cast<float2 *>(P.r)[j] = rv;
      reinterpret_cast<float4 *>(P.pz)[j] = make_float4(pz0.x, pz0.y, pz1.x, pz1.y);
    }
  } else {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < P.N && !is_fixed(Q, i)) {
      R2 pz = P.pz[i];
      R x = P.x[i], r = P.r[i];
      update_node(Q, i, alpha, beta, x, r, pz, P.q[i], P.dinv[i], vals, proj);
      P.x[i] = x;
      P.r[i] = r;
      P.pz[i] = pz;
    }
  }
  __shared__ double tot[3];
  const PlateC &c = B.pc[p];
  if (reduce_plate<R, 3>(vals, P.part, B.tick + p, c.blk0, c.nblk, tot) && threadIdx.x == 0) {
    Params<R> F = Q;
    F.use_cond = 0;
    update_finish(F, tot);
    plate_report(P, B, false);
  }
}

template <typename R>
__global__ void __launch_bounds__(256) kb_finish(Params<R> P, Batch B) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < P.N) {
    R v;
    if (P.flags[i] & kNotch) {
      v = R(1);
    } else {
      v = P.x[i];
      const R lo = P.dprev[i];
      v = v > lo ? v : lo;
      v = v < R(1) ? v : R(1);
    }
    P.dout[i] = v;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const int64_t n = *P.step_ctr;
    for (int q = 0; q < B.nplates; ++q) {
      const SolveScalars &S = B.sc[q];
      if (P.status_word && S.status) atomicMax(P.status_word, S.status);
      if (B.iters_log) B.iters_log[n * B.nplates + q] = S.iters;
    }
  }
}

// ------------------------------------------------ per-plate persistent CG
//
// Every plate's damage solve in one cooperative launch (a full wave of
// co-resident CTAs).  The CTAs are split into one group per plate, sized in
// proportion to the plate's rows (at least one each; cta0, ncta of
// PlateC).  A group runs k_cg_persistent's iteration on its own plate only:
// its rows are the plate's node blocks, its two all-reduces per iteration
// are among its own CTAs (the plate's barrier counter, the plate's slice of
// the partials, the group's rank order), it takes its plate's stop decision
// and leaves when its plate has converged -- the others go on.  Every wait
// is bounded as in the single-plate loop; a group that gives up marks only
// its plate (status timeout).  Same arithmetic per plate as the
// kernel-per-phase batch loop except for the grouping of the dot products'
// partial sums.
template <typename R, int U>
__global__ void __launch_bounds__(pers_threads(U, false), kPersMinBlocks) kb_cg_persistent(Params<R> P, Batch B) {
  typedef Acc<R> AC;
  const int2 gp = B.cta_plate[blockIdx.x];
  const int p = gp.x, rank = gp.y;
  Params<R> Q = P;
  plate_apply(Q, B, p);
  const PlateC &c = B.pc[p];
  SolveScalars *S = Q.sc;
  __shared__ typename AC::T sh[pers_threads(U, false) / 32][2];
  __shared__ PersShared<R> z;
  if (S->done) return;  // set-up found b_eff = 0 or r_0 already small
  if (threadIdx.x == 0) {
    pers_load(z, S, Q.tol);
    z.ok = 1;
  }
  __syncthreads();
  const unsigned int nb = (unsigned)c.ncta;
  const int n0 = c.blk0 * kThreadsBatch;
  const int n1 = min(P.N, (c.blk0 + c.nblk) * kThreadsBatch);
  const int T = (int)blockDim.x;
  const int tid = n0 + rank * T + (int)threadIdx.x, stride = (int)nb * T;
  // FP32 updates work in row pairs (n0 is even: plates start on 256-node blocks)
  const int pid = sizeof(R) == 4 ? n0 / 2 + rank * T + (int)threadIdx.x : tid;
  double *part = P.part + 4u * (unsigned)c.cta0;
  unsigned int nbar = 0;
  for (;;) {
    typename AC::T v1[1] = {AC::zero()};
    matvec_rows<R, U>(Q, z.coef[1], tid, stride, v1[0], n1, (z.iters & 1) != 0);
    ++nbar;
    if (!grid_sum<R, 1>(v1, part + (nbar & 1u) * 2u * nb, S, nbar * nb, z.tot, (typename AC::T(*)[1])sh, &z.ok,
                        NoHook(), rank, (int)nb))
      break;
    if (threadIdx.x == 0) {
      const bool moved = pers_alpha(z);  // p = 0: nothing moved, the iterate is exact
      z.done = moved ? z.done : 1;
      z.flag = moved ? 0 : 1;
    }
    __syncthreads();
    if (z.flag) break;
    typename AC::T v3[3] = {AC::zero(), AC::zero(), AC::zero()};
    bool proj = false;
    update_rows<R>(Q, z.coef[0], z.coef[1], pid, stride, v3, proj, n1, (z.iters & 1) != 0);
    typename AC::T v2[2] = {v3[0], v3[1]};
    ++nbar;
    if (!grid_sum<R, 2>(v2, part + (nbar & 1u) * 2u * nb, S, nbar * nb, z.tot, sh, &z.ok, NoHook(), rank,
                        (int)nb))
      break;
    if (threadIdx.x == 0) z.flag = pers_beta(z, Q.tol, P.max_it) ? 1 : 0;
    __syncthreads();
    if (z.flag) break;
  }
  // the group's first CTA leaves the plate's scalars as the phases loop would
  if (rank == 0 && threadIdx.x == 0) {
    pers_store(z, S);
    S->inner_done = 1;
  }
}

// ------------------------------------------------ per-plate resident CG
//
// k_cg_resident's single-reduction loop (FP32, fan-order rows, the partial
// form: x, p, the diagonal and the fan words of a CTA's rows in its shared
// memory) for many plates at once.  The plates are solved in waves, one
// cooperative launch each: a wave's plates together fit the SMs' shared
// memory, and their operator records and CG records (about 80 B a row)
// stay in L2 across the wave's iterations, where all plates at once would
// stream them from HBM every iteration.  Within a wave each plate has a
// group of CTAs, each owning a contiguous range of the plate's rows
// (ResCta); a group's all-reduces are among its own CTAs (the plate's
// barrier counter, its slice of the partials at the group's first CTA of
// the wave), it takes its plate's stop decision and leaves when its plate
// has converged.  Same arithmetic per row as k_cg_resident; the dot
// products' partial sums are grouped by CTA range.
struct ResCta {
  int32_t plate, rank;  // the plate, and the CTA's rank in the plate's group
  int32_t row0, nr;     // the CTA's rows [row0, row0 + nr)
  int32_t g0, ncta;     // the group's first CTA within the wave, and its size
};

template <int U>
__global__ void __launch_bounds__(res_threads(U), res_minb(U)) kb_cg_resident(Params<float> P, Batch B,
                                                                                const ResCta *map) {
  typedef Acc<float> AC;
  const ResCta c = map[blockIdx.x];
  Params<float> Q = P;
  plate_apply(Q, B, c.plate);
  SolveScalars *S = Q.sc;
  __shared__ DF sh[32][3];
  __shared__ FusedShared z;
  extern __shared__ __align__(16) uint32_t res_smem[];
  if (S->done) return;  // set-up found b_eff = 0 or r_0 already small
  const int R = P.res_rows, row0 = c.row0, nr = c.nr;
  float *xs = reinterpret_cast<float *>(res_smem);
  for (int l = threadIdx.x; l < nr; l += blockDim.x) {
    const int j = row0 + l;
    xs[l] = Q.x[j];
    xs[R + l] = 0.f;
    xs[2 * R + l] = Q.diag[j];
#pragma unroll
    for (int k = 0; k < 3; ++k) res_smem[(3 + k) * R + l] = __ldg(&Q.fno[(size_t)k * Q.N + j]);
    res_smem[6 * R + l] = (__ldg(&Q.fmap[j]) >> 24) | (is_fixed(Q, j) ? 0x100u : 0u);
    Q.cgv0[j] = make_float4(Q.r[j], 0.f, 0.f, Q.dinv[j]);
  }
  if (threadIdx.x == 0) fused_load(z, S, Q.tol);
  const unsigned int nb = (unsigned)c.ncta;
  double *part = P.part + 6u * (unsigned)c.g0;
  unsigned int nbar = 1;
  DF v3[3] = {AC::zero(), AC::zero(), AC::zero()};
  bool fine = grid_sum<float, 3>(v3, part + 3u * nb, S, nb, z.tot, sh, &z.ok, NoHook(), c.rank, (int)nb);
  int pass = 0;  // passes read cgv[pass & 1] and write the other buffer
  while (fine) {
    const float4 *vin = (pass & 1) ? Q.cgv1 : Q.cgv0;
    float4 *vout = (pass & 1) ? Q.cgv0 : Q.cgv1;
    DF acc[3] = {AC::zero(), AC::zero(), AC::zero()};
    resident_rows(Q, z.al, z.be, vin, vout, row0, nr, R, res_smem, acc, (pass & 1) != 0);
    ++nbar;
    ++pass;
    if (!grid_sum<float, 3>(acc, part + (nbar & 1u) * 3u * nb, S, nbar * nb, z.tot, sh, &z.ok, NoHook(), c.rank,
                            (int)nb))
      break;
    if (threadIdx.x == 0) fused_scalars(z, Q, pass);
    __syncthreads();
    if (z.flag) break;
  }
  for (int l = threadIdx.x; l < nr; l += blockDim.x) Q.x[row0 + l] = xs[l];
  if (c.rank == 0 && threadIdx.x == 0) fused_store(z, S);
}

// Advances the step counter after all kernels of the step read it.
__global__ void kb_step_done(int64_t *step_ctr) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *step_ctr += 1;
}

}  // namespace pff
