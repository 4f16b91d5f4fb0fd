// kernels.cuh -- device code of the phase-field fracture step for sm_103a.
//
// Force and damage-operator accumulation is a gather: every node sums the
// contributions of its incident elements (the node-to-element incidence,
// ascending element id), recomputing what it needs of each element from a
// packed 32-byte element record.  Accumulation is therefore a plain sum in a
// fixed order: no atomics, bit-identical reruns, and every schedule variant
// (entry-parallel node blocks or node-centric with U gathers in flight)
// adds the same terms in the same order.  Per-element results that must be
// stored once (the history H) are written by the element's slot-0 entry.
//
// The node-centric schedules read the incidence in ELL layout
// (entry j of node i at ell[j N + i], padded with -1), so that a warp's
// loads of one slot are coalesced.
//
// Precision.  R = double: everything FP64 (the parity mode).  R = float
// (FP32_MIXED): element and vector arithmetic in FP32; the history H stays
// FP64 and its max is taken exactly; inner products and norms are
// accumulated in double-word precision: each term is an exact FP32
// product (TwoProd), warps sum (hi, lo) pairs with TwoSum, and warps and
// blocks are summed in FP64.  B300 runs FP64 at ~1/57 of its FP32 rate, so
// per-node FP64 instructions would otherwise dominate every kernel.
//
// Reductions: each block writes one partial per value, and the last block
// to finish (ticket counter) sums the partials in block order.
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

// Packed element record: the three node ids, the area and the independent
// shape gradients (dphi0/dx, dphi0/dy, dphi1/dx, dphi1/dy) of Eq. (grad_phi);
// dphi2 = -(dphi0 + dphi1).  32 bytes (one sector) in FP32, 64 in FP64.
template <typename R> struct ERec;
template <> struct __align__(32) ERec<float> {
  int n0, n1, n2;
  float A;
  float4 g;
};
template <> struct __align__(64) ERec<double> {
  int n0, n1, n2, pad;
  double A, pad2;
  dbl4 g;
};

// Damage operator record of an element for one solve (the history is fixed
// while the damage CG runs): node ids, the off-diagonal stiffness weights
// w_ab = kappa_e A_e grad(phi_a) . grad(phi_b) and the mass coefficient
// mA = c_e A_e / 12 (Eqs. damage_pde_at2 / damage_pde_at1, consistent mass).
// Because the rows of the element stiffness sum to zero, row a of the
// element operator applied to x is
//   w_ab (x_b - x_a) + w_ac (x_c - x_a) + mA (2 x_a + x_b + x_c).
// 32 bytes (one sector) in FP32, 64 in FP64.
template <typename R> struct DRec;
template <> struct __align__(32) DRec<float> {
  int n0, n1, n2;
  float w01, w02, w12, mA, pad;
};
template <> struct __align__(64) DRec<double> {
  int n0, n1, n2, pad;
  double w01, w02, w12, mA;
};

// Scalars of one damage solve, living in device memory.  Dot products are
// of (rscale r), (rscale q) with z, p, so every ratio the solver uses is
// unchanged by the power-of-two scale.
struct SolveScalars {
  double bn;      // ||b - A 1_D|| over free rows (scaled)
  double rho;     // r . z
  double alpha, beta;
  double rr;      // ||r||^2 (free rows, scaled)
  double pq;
  int32_t iters, restarts, status, done;
  int32_t projected, inner_done;
  float alpha_f, beta_f;  // FP32 copies read by every thread in FP32 mode
  uint32_t bar;           // persistent CG: grid-barrier arrivals of this solve
  int32_t abort;          // persistent CG: a barrier wait gave up
};

// One CTA's share of the shared-memory staging: rows [row0, row1); element
// ranges [r0, r1) of the range table, nel elements in all, localized records
// at lrec; node ranges [n0, n1), nn nodes in all, of which row row0 is at
// position own.
struct StageCta {
  int32_t row0, row1, r0, r1, nel, lrec, n0, n1, nn, own;
};

// Everything a kernel needs, passed by value (graph-captured).
template <typename R> struct Params {
  typedef typename V<R>::T2 R2;
  typedef typename V<R>::T4 R4;
  int32_t N, Ne;
  int32_t NB, nblk;  // nodes per node block, number of node blocks
  int32_t D;         // ELL width (maximum incidence degree)
  // mesh
  const int32_t *__restrict__ ptr;
  const int32_t *__restrict__ ent;
  const int32_t *__restrict__ ell;
  const ERec<R> *__restrict__ rec;
  const uint8_t *__restrict__ flags;
  const R2 *__restrict__ fext;
  const R *__restrict__ minv;
  R2 *fe;  // 3 Ne: slot forces of the element-pass force schedule
  // operator staged in shared memory by the persistent CG (FP32), per CTA
  // (see StageCta): element ranges (first element, count), node ranges
  // (first node, count), element records with node ids replaced by node
  // positions in the CTA's staged node set, and the row entries: entry k of
  // row i at st_slot[k * st_ns + i] = position << 2 | a (0xffff: none)
  const StageCta *__restrict__ st_cta;
  const int2 *__restrict__ st_rng;
  const int2 *__restrict__ st_nrng;
  const ERec<float> *__restrict__ st_lrec;
  const uint16_t *__restrict__ st_slot;
  int32_t st_ns;
  // single-reduction CG (FP32): per node (r, w, s, 1/diag) in two buffers
  // (read one, write the other each pass) and the search direction p
  float4 *cgv0, *cgv1;
  float *cgp;
  int32_t res_rows;  // resident single-reduction CG: rows per CTA
  int32_t res_halo;  // its FULL form: the mesh's element span (bounds every neighbour offset)
  // material (lam: the plane model's first Lame parameter; K: 3-D bulk
  // modulus; cz = nu / (1 - nu) under plane stress, 0 under plane strain)
  R lam, mu, K, eta, cz;
  int32_t split, model;
  R kappa;      // damage diffusion coefficient (Gc l0 or 3/4 Gc l0)
  DRec<R> *drec; // damage records of the current solve (nullable: the
                 // operator is rebuilt from the geometry and H per entry);
                 // written by the right-hand-side kernels, read by the matvec
  float4 *erec;  // FP32: damage entry records of the current solve in the
                 // incidence layout (entry k of node i at k N + i): the other
                 // two nodes b, c of the entry's element and their row
                 // coefficients (w_ab + mA, w_ac + mA); b = -1 marks an empty
                 // slot.  Nullable.
  uint32_t *ecmp; // compact form of the same (meshes whose elements span
  float2 *ecf;    // fewer than 2^15 node ids): ecmp packs the 16-bit offsets
                  // b - i (low half) and c - i (high half), ecf the two
                  // coefficients; an empty slot is offsets 0, coefficients 0.
                  // Nullable; at most one of erec and ecmp is set.
  double2 *ecfd;  // FP64 meshes: the entry coefficients in FP64 (with ecmp)
  // Fan order (compact meshes whose every vertex fan fits six positions):
  // fno packs the row's distinct neighbours v_0..v_{m-1} as 16-bit offsets
  // in counter-clockwise order around the vertex (three words, layout
  // w N + i, zero padded); fmap[i] holds m in its top byte and, in 4-bit
  // fields, the fan position of each incidence slot.  With them the entry
  // records are stored in fan position (the fan's k-th triangle couples
  // v_k and v_{k+1 mod m}, its two coefficients in that order) and a row
  // gathers each distinct neighbour once.  Nullable.
  const uint32_t *__restrict__ fno;
  const uint32_t *__restrict__ fmap;
  // Compact meshes (both precisions) whose rows have at most kNbMax distinct
  // neighbours:
  // the same rows with each neighbour's coefficients merged (rows sum the
  // per-element coefficients of a neighbour shared by two elements once):
  // nbo packs the row's ascending neighbour offsets j - i two per word
  // (Dn / 2 words, incidence-style layout w N + i), nbc holds the merged
  // coefficient of each (Dn x N); padding slots are offset 0, coefficient
  // 0.  nmap (one 8-byte word per row, byte k for incidence slot k) gives
  // the merged slots of the entry's two neighbours (low and high nibble;
  // 0xff = empty).  The right-hand side fills nbc.  Nullable.
  const uint32_t *__restrict__ nbo;
  R *nbc;
  const uint2 *__restrict__ nmap;
  int32_t Dn;
  // Element-wise form (FP32 compact records, rows with at most six
  // incidence slots and six distinct neighbours): the same offset words
  // and slot maps, used only to gather each distinct neighbour's value
  // once per row; every entry still applies its own element's two
  // coefficients (ecf).  Nullable (then each slot gathers its two nodes).
  const uint32_t *__restrict__ gnbo;
  const uint2 *__restrict__ gmap;
  R *diag;       // with erec: the row's diagonal sum over entries of
                 // (kappa_e A_e |grad phi_a|^2 + 2 mA)
  const R *gcs; // per-element toughness field as Gc_e / Gc (nullable: uniform);
                // kappa, cbase and wbase are linear in Gc and scale with it
  R cbase;      // reaction: c_e = cbase + 2 H_e
  R wbase;      // load:     w_e = wbase + 2 H_e
  R rscale;     // power of two applied to residual-like vectors in the dots
  double Gc, l0;
  // state
  R2 *u, *v, *a;
  R *d;
  double *H;         // history (always FP64)
  const R *Hr;       // history in the kernel precision (H itself, or Hf)
  float *Hf;         // FP32 mirror of H kept by k_force (FP32 mode only)
  // time and load: the traction scale S(t) of Eq. (smooth_traction_ramp)
  // is evaluated on the host.  Single step: S_prev = S(t_n), S_next =
  // S(t_n+1).  Graph-run steps: Stab[k] = S(t_{n0+k}) for the run's k-th
  // step, k read from the device counter step_ctr.
  double dt, t_ramp;
  double S_prev, S_next;
  const double *Stab;
  const int64_t *step_ctr;
  // damage solve
  const R *dprev;
  R *dout;
  R *x, *r, *b;
  R2 *pz;      // (p, z) interleaved: search direction and preconditioned residual
  R *q, *dinv;
  uint8_t *freef;
  double *part;
  unsigned int *ticket;
  SolveScalars *sc;
  double tol;
  int32_t max_it, max_restarts;
  int32_t use_cond;
  int32_t bar_extra;  // persistent CG: arrivals awaited beyond the grid (0; 1 = test of the bounded wait)
  cudaGraphConditionalHandle cond_inner, cond_outer;
  // logs
  int32_t *iters_log;     // device, per step (iters, restarts)
  int32_t *status_word;   // device, worst status (atomicMax)
  int64_t *step_inc;      // counter incremented at the end of a step
  double *energy_out;     // 4 doubles: E_el, E_kin, E_frac, W_ext
  double *wext;           // running external work
  int32_t track_work;
};

// ------------------------------------------------------- accumulators

// Unevaluated sum hi + lo of two floats (double-word arithmetic).
struct DF {
  float hi, lo;
};

// Exact product a*b = hi + lo (TwoProd with an FMA).
__device__ __forceinline__ DF two_prod(float a, float b) {
  const float p = a * b;
  return DF{p, fmaf(a, b, -p)};
}

// Double-word addition: TwoSum of the high parts, then the low parts.
__device__ __forceinline__ DF df_add(DF a, DF b) {
  const float s = a.hi + b.hi;
  const float bb = s - a.hi;
  float e = (a.hi - (s - bb)) + (b.hi - bb);
  e += a.lo + b.lo;
  const float hi = s + e;
  return DF{hi, e - (hi - s)};
}

// Double-word arithmetic for the single-reduction loops' scalar step, in
// FP32 instructions only (an FP64 warp instruction costs ~17 SM cycles on
// this GPU, and the step is on every iteration's critical path).  Products
// and quotients of (hi, lo) pairs after Dekker (1971), in the forms whose
// errors Joldes, Muller and Popescu (2017) bound by a few units of 2^-44
// relative: ample for alpha and beta, which the rows use rounded to FP32.
__device__ __forceinline__ DF df_fast(float a, float b) {  // |a| >= |b| or a = 0
  const float s = a + b;
  return DF{s, b - (s - a)};
}
__device__ __forceinline__ DF df_mul(DF a, DF b) {
  const DF p = two_prod(a.hi, b.hi);
  return df_fast(p.hi, p.lo + fmaf(a.hi, b.lo, a.lo * b.hi));
}
__device__ __forceinline__ DF df_div(DF a, DF b) {
  const float q1 = a.hi / b.hi;
  const DF qb = df_mul(DF{q1, 0.f}, b);
  const DF r = df_add(a, DF{-qb.hi, -qb.lo});
  return df_fast(q1, r.hi / b.hi);
}
__device__ __forceinline__ DF df_sub(DF a, DF b) { return df_add(a, DF{-b.hi, -b.lo}); }
__device__ __forceinline__ bool df_le(DF a, DF b) { return a.hi < b.hi || (a.hi == b.hi && a.lo <= b.lo); }
__device__ __forceinline__ bool df_finite(DF a) { return isfinite(a.hi) && isfinite(a.lo); }
__device__ __forceinline__ DF df_from(double d) {
  const float hi = (float)d;
  return DF{hi, (float)(d - (double)hi)};
}
__device__ __forceinline__ double df_to(DF a) { return (double)a.hi + (double)a.lo; }

template <typename R> struct Acc;
template <> struct Acc<double> {
  typedef double T;
  static __device__ __forceinline__ T zero() { return 0.0; }
  static __device__ __forceinline__ T prod(double a, double b) { return a * b; }
  static __device__ __forceinline__ T add(T a, T b) { return a + b; }
  static __device__ __forceinline__ T shfl(T v, int o) { return __shfl_down_sync(0xffffffffu, v, o); }
  static __device__ __forceinline__ double to_d(T v) { return v; }
  static __device__ __forceinline__ T one() { return 1.0; }
  static __device__ __forceinline__ void store(double *p, T v) { *p = v; }
  static __device__ __forceinline__ T load(const double *p) { return __ldcg(p); }
};
template <> struct Acc<float> {
  typedef DF T;
  static __device__ __forceinline__ T zero() { return DF{0.f, 0.f}; }
  static __device__ __forceinline__ T prod(float a, float b) { return two_prod(a, b); }
  static __device__ __forceinline__ T add(T a, T b) { return df_add(a, b); }
  static __device__ __forceinline__ T shfl(T v, int o) {
    return DF{__shfl_down_sync(0xffffffffu, v.hi, o), __shfl_down_sync(0xffffffffu, v.lo, o)};
  }
  static __device__ __forceinline__ double to_d(T v) { return (double)v.hi + (double)v.lo; }
  static __device__ __forceinline__ T one() { return DF{1.f, 0.f}; }
  static __device__ __forceinline__ void store(double *p, T v) {
    *reinterpret_cast<float2 *>(p) = make_float2(v.hi, v.lo);
  }
  static __device__ __forceinline__ T load(const double *p) {
    const float2 f = __ldcg(reinterpret_cast<const float2 *>(p));
    return DF{f.x, f.y};
  }
};

// Block-reduces NV accumulators, publishes one partial per block and
// returns true in every thread of the last block to arrive; that block then
// finds the totals (converted to FP64) in `tot` (shared).  The whole
// reduction stays in the accumulator type (double-word FP32 in FP32 mode:
// B300 issues an FP64 warp instruction in ~17 SM cycles), with one
// conversion at the end.  Fixed summation order.
template <typename R, int NV>
__device__ __forceinline__ bool reduce_last(typename Acc<R>::T (&v)[NV], double *part,
                                            unsigned int *ticket, double *tot) {
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
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  // the last block sums the partials: thread j takes blocks j, j+B, ...;
  // eight loads are issued before they are added (one L2 round trip each)
  T acc[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    acc[k] = A::zero();
    for (int j0 = threadIdx.x; j0 < (int)gridDim.x; j0 += 8 * blockDim.x) {
      T buf[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int j = j0 + u * blockDim.x;
        buf[u] = j < (int)gridDim.x ? A::load(&part[(size_t)j * NV + k]) : A::zero();
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

// CG coefficients in the kernel precision (FP32 copies in FP32 mode, so no
// thread converts from FP64).
template <typename R> __device__ __forceinline__ R sc_alpha(const SolveScalars *S) {
  return sizeof(R) == 4 ? (R)S->alpha_f : (R)S->alpha;
}
template <typename R> __device__ __forceinline__ R sc_beta(const SolveScalars *S) {
  return sizeof(R) == 4 ? (R)S->beta_f : (R)S->beta;
}

template <typename R> __device__ __forceinline__ R rpos(R x) { return x > R(0) ? x : R(0); }

// Element e's toughness relative to the material's (1 without a field).
template <typename R> __device__ __forceinline__ R gc_scale(const Params<R> &P, int e) {
  return P.gcs ? P.gcs[e] : R(1);
}
template <typename R> __device__ __forceinline__ R rneg(R x) { return x < R(0) ? x : R(0); }

// Accumulation a + b that the compiler may not contract into an FMA with
// the producer of b: every schedule then rounds the same sums the same way.
__device__ __forceinline__ float radd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double radd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float rfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double rfma(double a, double b, double c) { return __fma_rn(a, b, c); }

// Load scale at the end (which = 1) or start (which = 0) of the step.
template <typename R>
__device__ __forceinline__ double load_scale(const Params<R> &P, int which) {
  if (P.step_ctr) return P.Stab[*P.step_ctr + which];
  return which ? P.S_next : P.S_prev;
}

// IEEE-754 bit pattern of the double equal to a non-negative float (exact
// conversion done with integer instructions; subnormal floats give 0).
// Non-negative doubles order like their bit patterns, so the history max
// max(H, psi+) is decided exactly without FP64 instructions.
__device__ __forceinline__ long long f2d_bits(float f) {
  const unsigned int b = __float_as_uint(f);
  const unsigned int ex = (b >> 23) & 0xffu;
  if (ex == 0u || (b >> 31)) return 0;
  return ((long long)(ex - 127u + 1023u) << 52) | ((long long)(b & 0x7fffffu) << 29);
}

// Degraded stress and psi+ at one element (tensor strain components).
// Spectral (Eq. spectral_split): with D = eps - tr/2 I and R = |D|, the
// tensile part is eps+ = (<e1>+ + <e2>+)/2 I + (<e1>+ - <e2>+)/(2R) D.
// Volumetric-deviatoric (Eq. amor_split) uses the 3-D deviator of the
// strain with e_zz = -cz tr (0 in plane strain; plane stress: the
// out-of-plane strain of Sec. 2.1, whose dependence on the in-plane strain
// enters the stress).  sigma = g sigma+ + sigma-.
// Every multiply-add is written out (rfma / rmul / radd): which products
// the compiler would fuse otherwise depends on the code around the call
// (how often each product is used there), and the kernels that evaluate an
// element once per incidence entry and those that evaluate it once per
// element must round alike.
template <typename R>
__device__ __forceinline__ void stress(const Params<R> &P, R exx, R eyy, R exy, R g,
                                       R &sxx, R &syy, R &sxy, R &psip) {
  const R tr = radd(exx, eyy);
  const R trp = rpos(tr), trm = rneg(tr);
  // exx^2 + eyy^2 + 2 exy^2
  const R sq = rfma(rmul(R(2), exy), exy, rfma(exx, exx, rmul(eyy, eyy)));
  if (P.split == kSpectral) {
    const R half = rmul(R(0.5), exx - eyy);
    const R rad = sqrt(rfma(half, half, rmul(exy, exy)));
    const R e1 = rfma(R(0.5), tr, rad), e2 = rfma(R(0.5), tr, -rad);
    const R e1p = rpos(e1), e2p = rpos(e2);
    const R s = rad > R(0) ? (e1p - e2p) / rmul(R(2), rad) : R(0);
    const R m = rmul(R(0.5), radd(e1p, e2p));
    const R pxx = rfma(s, half, m), pyy = rfma(-s, half, m), pxy = rmul(s, exy);
    const R tm = rmul(P.lam, trm), tp = rmul(P.lam, trp), mu2 = rmul(R(2), P.mu);
    sxx = rfma(mu2, exx - pxx, rfma(g, rfma(mu2, pxx, tp), tm));
    syy = rfma(mu2, eyy - pyy, rfma(g, rfma(mu2, pyy, tp), tm));
    sxy = rfma(g, rmul(mu2, pxy), rmul(mu2, exy - pxy));
    psip = rfma(P.mu, rfma(e1p, e1p, rmul(e2p, e2p)), rmul(rmul(rmul(R(0.5), P.lam), trp), trp));
  } else if (P.split == kAmor && P.cz == R(0)) {
    const R t3 = rmul(tr, R(1) / R(3)), mu2 = rmul(R(2), P.mu), km = rmul(P.K, trm);
    sxx = rfma(g, rfma(P.K, trp, rmul(mu2, exx - t3)), km);
    syy = rfma(g, rfma(P.K, trp, rmul(mu2, eyy - t3)), km);
    sxy = rmul(g, rmul(mu2, exy));
    psip = rfma(P.mu, rfma(-tr, t3, sq), rmul(rmul(rmul(R(0.5), P.K), trp), trp));
  } else if (P.split == kAmor) {
    // plane stress: e_zz = -cz tr, tr3 = f tr with f = 1 - cz; the in-plane
    // stresses carry d e_zz / d e_ii = -cz
    const R f = R(1) - P.cz, ez = rmul(-P.cz, tr), tr3 = rmul(f, tr);
    const R t3p = rpos(tr3), t3m = rneg(tr3), mu2 = rmul(R(2), P.mu), kf = rmul(P.K, f);
    const R lin = rfma(rmul(P.cz, P.cz), tr, -rmul(rmul(f, tr3), R(1) / R(3)));
    sxx = rfma(g, rfma(kf, t3p, rmul(mu2, radd(exx, lin))), rmul(kf, t3m));
    syy = rfma(g, rfma(kf, t3p, rmul(mu2, radd(eyy, lin))), rmul(kf, t3m));
    sxy = rmul(g, rmul(mu2, exy));
    psip = rfma(P.mu, rfma(-rmul(tr3, tr3), R(1) / R(3), rfma(ez, ez, sq)),
                rmul(rmul(rmul(R(0.5), P.K), t3p), t3p));
  } else {
    const R mu2 = rmul(R(2), P.mu);
    sxx = rmul(g, rfma(P.lam, tr, rmul(mu2, exx)));
    syy = rmul(g, rfma(P.lam, tr, rmul(mu2, eyy)));
    sxy = rmul(g, rmul(mu2, exy));
    psip = rfma(P.mu, sq, rmul(rmul(rmul(R(0.5), P.lam), tr), tr));
  }
}

template <typename R, typename R4>
__device__ __forceinline__ void slot_grad(const R4 &G, int a, R &gx, R &gy) {
  gx = a == 0 ? G.x : (a == 1 ? G.z : -(G.x + G.z));
  gy = a == 0 ? G.y : (a == 1 ? G.w : -(G.y + G.w));
}

template <typename R>
__device__ __forceinline__ bool is_fixed(const Params<R> &P, int i) {
  return (P.flags[i] & kNotch) || (P.freef && !P.freef[i]);
}

// ------------------------------------------------------------ mechanics
//
// Node-block kernels: block b owns nodes [b NB, (b+1) NB) and walks all
// their incidence entries [ptr[i0], ptr[i1]) with one thread per entry
// (independent gathers, high memory-level parallelism); each entry's
// contribution is staged in shared memory, then one thread per node sums
// its own entries in ascending element order.

template <typename R>
__device__ __forceinline__ void block_nodes(const Params<R> &P, int b, int &i0, int &i1, int &k0, int &k1) {
  i0 = b * P.NB;
  i1 = min(i0 + P.NB, P.N);
  k0 = __ldg(&P.ptr[i0]);
  k1 = __ldg(&P.ptr[i1]);
}

// Loads element e's record: node ids, area and shape gradients.  The FP32
// record is one 32-byte sector, read with a single 256-bit load.
template <typename R>
__device__ __forceinline__ void load_elem(const Params<R> &P, int e, int4 &t, R &A,
                                          typename Params<R>::R4 &G) {
  const ERec<R> *rp = P.rec + e;
  if (sizeof(R) == 4) {
    unsigned w0, w1, w2, w3, w4, w5, w6, w7;
    asm("ld.global.nc.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=r"(w0), "=r"(w1), "=r"(w2), "=r"(w3), "=r"(w4), "=r"(w5), "=r"(w6), "=r"(w7)
        : "l"(rp));
    t = make_int4((int)w0, (int)w1, (int)w2, 0);
    A = (R)__uint_as_float(w3);
    G.x = (R)__uint_as_float(w4);
    G.y = (R)__uint_as_float(w5);
    G.z = (R)__uint_as_float(w6);
    G.w = (R)__uint_as_float(w7);
  } else {
    t = __ldg(reinterpret_cast<const int4 *>(rp));
    const double2 a = __ldg(reinterpret_cast<const double2 *>(rp) + 1);
    const double2 g0 = __ldg(reinterpret_cast<const double2 *>(rp) + 2);
    const double2 g1 = __ldg(reinterpret_cast<const double2 *>(rp) + 3);
    A = (R)a.x;
    G.x = (R)g0.x; G.y = (R)g0.y; G.z = (R)g1.x; G.w = (R)g1.y;
  }
}

// Strain (tensor components) of an element from its three nodes' u.
template <typename R, typename R2, typename R4>
__device__ __forceinline__ void elem_strain_u(const R4 &G, const R2 &u0, const R2 &u1, const R2 &u2,
                                              R &exx, R &eyy, R &exy) {
  const R ax0 = u0.x - u2.x, ax1 = u1.x - u2.x, ay0 = u0.y - u2.y, ay1 = u1.y - u2.y;
  exx = rfma(G.x, ax0, rmul(G.z, ax1));
  eyy = rfma(G.y, ay0, rmul(G.w, ay1));
  exy = rmul(R(0.5), rfma(G.z, ay1, rfma(G.x, ay0, rfma(G.y, ax0, rmul(G.w, ax1)))));
}

// Strain (tensor components) of element e from nodal u.
template <typename R>
__device__ __forceinline__ void elem_strain(const Params<R> &P, const typename Params<R>::R4 &G, const int4 &t,
                                            R &exx, R &eyy, R &exy) {
  typedef typename Params<R>::R2 R2;
  const R2 u0 = P.u[t.x], u1 = P.u[t.y], u2 = P.u[t.z];
  elem_strain_u<R>(G, u0, u1, u2, exx, eyy, exy);
}

// Predictor, Eq. (vv_u): u += dt v + dt^2/2 a.  With track_work the
// trapezoid-rule external work increment 1/2 (S_n + S_n+1) f_ext . du is
// reduced into *wext.
template <typename R>
__global__ void __launch_bounds__(256) k_predict(Params<R> P) {
  typedef typename Params<R>::R2 R2;
  constexpr int B = 4;  // nodes per thread and pass: every load issued before the first store
  double w = 0.0;
  const int stride = gridDim.x * blockDim.x;
  const R dt = (R)P.dt, h = R(0.5) * dt * dt;
  for (int i0 = blockIdx.x * blockDim.x + threadIdx.x; i0 < P.N; i0 += B * stride) {
    R2 u[B], v[B], a[B];
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const int i = i0 + b * stride;
      if (i < P.N) {
        u[b] = P.u[i];
        v[b] = P.v[i];
        a[b] = P.a[i];
      }
    }
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const int i = i0 + b * stride;
      if (i >= P.N) break;
      const R dux = dt * v[b].x + h * a[b].x, duy = dt * v[b].y + h * a[b].y;
      if (P.track_work && (P.flags[i] & kLoaded)) {
        const double S = 0.5 * (load_scale(P, 0) + load_scale(P, 1));
        const R2 f = P.fext[i];
        w += S * ((double)f.x * dux + (double)f.y * duy);
      }
      u[b].x += dux;
      u[b].y += duy;
      P.u[i] = u[b];
    }
  }
  if (P.track_work) {
    double v1[1] = {w};
    __shared__ double tot[1];
    if (reduce_last<double, 1>(v1, P.part, P.ticket, tot) && threadIdx.x == 0) *P.wext += tot[0];
  }
}

// f_a = A (sigma . grad(phi_a)) with every rounding spelled out, so that a
// slot known at compile time (element pass) and one selected at run time
// (per-entry schedules) give the same bits.
template <typename R>
__device__ __forceinline__ void slot_force(R A, R sxx, R syy, R sxy, R gx, R gy, R &fx, R &fy) {
  fx = rmul(A, rfma(sxx, gx, rmul(sxy, gy)));
  fy = rmul(A, rfma(sxy, gx, rmul(syy, gy)));
}

// Force contribution of one incidence entry (element e at local slot a):
// f_a = A_e sigma_e . grad(phi_a) with sigma = g(dbar) sigma+ + sigma-
// (Sec. 2.3 gather and element contraction); also returns psi+_e.
template <typename R>
__device__ __forceinline__ void force_entry(const Params<R> &P, int en, R &fx, R &fy, R &psip) {
  typedef typename Params<R>::R4 R4;
  const int e = en >> 2, a = en & 3;
  int4 t;
  R A;
  R4 G;
  load_elem(P, e, t, A, G);
  R exx, eyy, exy;
  elem_strain(P, G, t, exx, eyy, exy);
  const R db = rmul(radd(radd(P.d[t.x], P.d[t.y]), P.d[t.z]), R(1) / R(3));
  const R g = rfma(R(1) - db, R(1) - db, P.eta);
  R sxx, syy, sxy;
  stress(P, exx, eyy, exy, g, sxx, syy, sxy, psip);
  R gx, gy;
  slot_grad<R>(G, a, gx, gy);
  slot_force(A, sxx, syy, sxy, gx, gy, fx, fy);
}

// History update H_e = max(H_e, psi+_e) by the element's owner entry
// (slot 0), Sec. 2.2.  FP32 mode decides the FP64 max on bit patterns
// (exact) and keeps the FP32 mirror equal to (float) H.
template <typename R>
__device__ __forceinline__ void history_update(const Params<R> &P, int en, R psip) {
  if (en & 3) return;
  const int e = en >> 2;
  if (sizeof(R) == 8) {
    const double hp = (double)psip;
    if (hp > P.H[e]) P.H[e] = hp;
  } else {
    const long long pb = f2d_bits((float)psip);
    const long long hb = __double_as_longlong(P.H[e]);
    if (pb > hb) {
      P.H[e] = __longlong_as_double(pb);
      P.Hf[e] = (float)psip;
    }
  }
}

// Acceleration and corrector at node i from its summed internal force,
// Eqs. (vv_a), (vv_v).
template <typename R>
__device__ __forceinline__ void corrector(const Params<R> &P, int i, R fx, R fy, double S) {
  typedef typename Params<R>::R2 R2;
  R Sf = 0, fex = 0, fey = 0;
  if (P.flags[i] & kLoaded) {
    Sf = (R)S;
    const R2 fe = P.fext[i];
    fex = fe.x;
    fey = fe.y;
  }
  const R mi = P.minv[i];
  const R anx = rmul(mi, rfma(Sf, fex, -fx)), any = rmul(mi, rfma(Sf, fey, -fy));
  R2 v = P.v[i], ao = P.a[i];
  const R hd = rmul(R(0.5), (R)P.dt);
  v.x = rfma(hd, radd(ao.x, anx), v.x);
  v.y = rfma(hd, radd(ao.y, any), v.y);
  P.v[i] = v;
  R2 an;
  an.x = anx;
  an.y = any;
  P.a[i] = an;
}

// Internal force at u_{n+1} with d_n, history, acceleration and corrector.
// Entry-parallel schedule (node blocks, contributions staged in shared
// memory, per-node sums in ascending element order).
// Force schedule "element pass + gather": one thread per element computes
// the strain, split and degraded stress once, updates the element's history
// and writes the three slot forces (force_entry's arithmetic); then one
// thread per node sums its slot forces in incidence order (the node-centric
// schedules' order, so all schedules give the same bits) and applies the
// corrector.
template <typename R>
__global__ void __launch_bounds__(256) k_force_elem(Params<R> P) {
  typedef typename Params<R>::R2 R2;
  typedef typename Params<R>::R4 R4;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < P.Ne; e += gridDim.x * blockDim.x) {
    int4 t;
    R A;
    R4 G;
    load_elem(P, e, t, A, G);
    R exx, eyy, exy;
    elem_strain(P, G, t, exx, eyy, exy);
    const R db = rmul(radd(radd(P.d[t.x], P.d[t.y]), P.d[t.z]), R(1) / R(3));
    const R g = rfma(R(1) - db, R(1) - db, P.eta);
    R sxx, syy, sxy, psip;
    stress(P, exx, eyy, exy, g, sxx, syy, sxy, psip);
    history_update(P, e << 2, psip);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      R gx, gy;
      slot_grad<R>(G, a, gx, gy);
      R2 f;
      slot_force(A, sxx, syy, sxy, gx, gy, f.x, f.y);
      P.fe[(size_t)3 * e + a] = f;
    }
  }
}

template <typename R>
__global__ void __launch_bounds__(256) k_force_gather(Params<R> P) {
  typedef typename Params<R>::R2 R2;
  const double S = load_scale(P, 1);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.N; i += gridDim.x * blockDim.x) {
    R fx = 0, fy = 0;
    for (int k = 0; k < P.D; k += 4) {
      int en[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) en[u] = k + u < P.D ? __ldg(&P.ell[(size_t)(k + u) * P.N + i]) : -1;
      R2 f[4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (en[u] >= 0) f[u] = P.fe[(size_t)3 * (en[u] >> 2) + (en[u] & 3)];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (en[u] >= 0) {
          fx = radd(fx, f[u].x);
          fy = radd(fy, f[u].y);
        }
    }
    corrector(P, i, fx, fy, S);
  }
}

// Same computation, node-centric schedule: one thread per node walks its
// entries U at a time with all U gathers issued before use (independent
// load chains); sums in the same ascending order, so the result is
// bit-identical to the entry-parallel schedule.
// FP32: at most 40 registers, so that six blocks share an SM (the gather is
// latency-bound: more warps in flight hide more of it).
template <typename R, int U>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 6 : 1) k_force_nc(Params<R> P) {
  const double S = load_scale(P, 1);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.N; i += gridDim.x * blockDim.x) {
    R fx = 0, fy = 0;
    for (int k = 0; k < P.D; k += U) {
      int en[U];
      R cx[U], cy[U], pp[U];
#pragma unroll
      for (int u = 0; u < U; ++u) en[u] = k + u < P.D ? __ldg(&P.ell[(size_t)(k + u) * P.N + i]) : -1;
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (en[u] >= 0) force_entry(P, en[u], cx[u], cy[u], pp[u]);
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (en[u] >= 0) {
          fx = radd(fx, cx[u]);
          fy = radd(fy, cy[u]);
          history_update(P, en[u], pp[u]);
        }
    }
    corrector(P, i, fx, fy, S);
  }
}

// FP32 mirror of the history: Hf = (float) H.
__global__ void k_h_mirror(const double *H, float *Hf, int n) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) Hf[e] = (float)H[e];
}

// --------------------------------------------------------------- damage

// Element contribution to row `a` of A x for element coefficients kA =
// kappa A_e, mA = c_e A_e / 12 (consistent mass, Sec. 2.4):
//   kA grad(phi_a) . grad(x_e) + mA (x_a + x_0 + x_1 + x_2).
template <typename R, typename R4>
__device__ __forceinline__ R elem_row(const R4 &G, int a, R kA, R mA, R x0, R x1, R x2) {
  const R dx = rfma(G.x, x0 - x2, rmul(G.z, x1 - x2));
  const R dy = rfma(G.y, x0 - x2, rmul(G.w, x1 - x2));
  R gx, gy;
  slot_grad<R>(G, a, gx, gy);
  const R xa = a == 0 ? x0 : (a == 1 ? x1 : x2);
  return rfma(kA, rfma(gx, dx, rmul(gy, dy)), rmul(mA, radd(radd(radd(xa, x0), x1), x2)));
}

// Entry record of slot a of an element (FP32 entry records): the other two
// nodes b, c and the coefficients of their values in row a,
//   kA grad(phi_a) . grad(phi_b) + mA  and  kA grad(phi_a) . grad(phi_c) + mA,
// the row's own coefficient kA |grad(phi_a)|^2 + 2 mA going to the diagonal
// (the element stiffness rows sum to zero, so row a of the element operator
// is exactly this split).
template <typename R>
__device__ __forceinline__ bool has_erec(const Params<R> &P) {
  return P.erec != nullptr || P.ecmp != nullptr;
}

// Writes the coefficients of the entry record of slot a of an element at
// (slot k, node i); the neighbour ids or offsets depend on the mesh alone
// and are written once (k_erec_ids).
template <typename R>
__device__ __forceinline__ typename Params<R>::R2 erec_coef(const typename Params<R>::R4 &G, int a, R kA, R mA,
                                                            bool ccw = false) {
  R gx, gy, gbx, gby, gcx, gcy;
  slot_grad<R>(G, a, gx, gy);
  // (b, c): the element's other slots in increasing order, or
  // counter-clockwise from a ((a+1, a+2) mod 3)
  const int sb = ccw ? (a == 2 ? 0 : a + 1) : (a == 0 ? 1 : 0);
  const int sc = ccw ? (a == 0 ? 2 : a - 1) : (a == 2 ? 1 : 2);
  slot_grad<R>(G, sb, gbx, gby);
  slot_grad<R>(G, sc, gcx, gcy);
  typename Params<R>::R2 c;  // roundings spelled out: every schedule gets the same bits
  c.x = rfma(kA, rfma(gx, gbx, rmul(gy, gby)), mA);
  c.y = rfma(kA, rfma(gx, gcx, rmul(gy, gcy)), mA);
  return c;
}

// Fan word of row i for put_erec (kFanLoad: put_erec reads it itself).
constexpr uint32_t kFanLoad = 0xffffffffu;
template <typename R>
__device__ __forceinline__ uint32_t fan_word(const Params<R> &P, int i) {
  return P.fmap ? __ldg(&P.fmap[i]) : 0u;
}

template <typename R>
__device__ __forceinline__ void put_erec(const Params<R> &P, int k, int i, const typename Params<R>::R4 &G, int a,
                                         R kA, R mA, uint32_t fm = kFanLoad) {
  // fan order: at the fan position of incidence slot k, the pair ordered
  // (v_k, v_{k+1}), counter-clockwise from the vertex
  const bool fan = P.fmap != nullptr;
  const typename Params<R>::R2 cr = erec_coef<R>(G, a, kA, mA, fan);
  size_t q = (size_t)k * P.N + i;
  if (fan) {
    if (fm == kFanLoad) fm = __ldg(&P.fmap[i]);
    q = (size_t)((fm >> (4 * k)) & 15u) * P.N + i;
  }
  if constexpr (sizeof(R) == 8) {
    if (P.ecfd) P.ecfd[q] = make_double2((double)cr.x, (double)cr.y);
    return;
  }
  const float2 c = make_float2((float)cr.x, (float)cr.y);
  if (P.ecmp)
    P.ecf[q] = c;
  else
    reinterpret_cast<float2 *>(P.erec + q)[1] = c;
}

// The mesh-only half of the entry records, once per mesh: per incidence
// slot the other two nodes of the entry's element (16-bit offsets from the
// row packed in one word, or the ids in the 16-byte form); empty slots get
// offsets 0 (or ids -1).  Coefficients start at 0.
template <typename R>
__global__ void __launch_bounds__(256) k_erec_ids(const ERec<R> *rec, const int *ell, int N, int D, uint32_t *ecmp,
                                                  float4 *erec) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    for (int k = 0; k < D; ++k) {
      const size_t q = (size_t)k * N + i;
      const int en = __ldg(&ell[q]);
      int nb = -1, nc = -1;
      if (en >= 0) {
        const ERec<R> &r = rec[en >> 2];
        const int a = en & 3;
        nb = a == 0 ? r.n1 : r.n0;
        nc = a == 2 ? r.n1 : r.n2;
      }
      if (ecmp)
        ecmp[q] = en < 0 ? 0u : ((uint32_t)(uint16_t)(int16_t)(nb - i) | ((uint32_t)(uint16_t)(int16_t)(nc - i) << 16));
      else
        erec[q] = make_float4(__int_as_float(nb), __int_as_float(nc), 0.f, 0.f);
    }
  }
}

constexpr int kNbMax = 8;  // merged rows: most distinct neighbours of a row

// The mesh-only half of the merged rows, once per mesh (compact records):
// per node the distinct neighbour offsets of its incidence entries in
// ascending order.  With maxcnt the largest count goes there (one atomic
// max per warp); else the offsets (Dn slots, padded with 0) and each
// incidence slot's merged slots are written.
__global__ void __launch_bounds__(256) k_nb_build(const uint32_t *__restrict__ ecmp, int N, int D, int Dn,
                                                  int *maxcnt, uint32_t *nbo, uint2 *nmap) {
  int most = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    int o[2 * kNbMax];
    int n = 0;
    for (int k = 0; k < D && k < kNbMax; ++k) {
      const uint32_t w = ecmp[(size_t)k * N + i];
      if (w == 0u) continue;  // empty slot (a real neighbour is never at offset 0)
      const int c2[2] = {(int)(int16_t)(w & 0xffffu), (int)w >> 16};
      for (int h = 0; h < 2; ++h) {
        int j = 0;
        while (j < n && o[j] < c2[h]) ++j;
        if (j < n && o[j] == c2[h]) continue;
        for (int m = n; m > j; --m) o[m] = o[m - 1];
        o[j] = c2[h];
        ++n;
      }
    }
    if (maxcnt) {
      most = max(most, D > kNbMax ? 2 * kNbMax : n);
      continue;
    }
    for (int w = 0; w < Dn / 2; ++w) {
      const int lo = 2 * w < n ? o[2 * w] : 0, hi = 2 * w + 1 < n ? o[2 * w + 1] : 0;
      nbo[(size_t)w * N + i] = (uint32_t)(uint16_t)(int16_t)lo | ((uint32_t)(uint16_t)(int16_t)hi << 16);
    }
    uint32_t mw[2] = {0xffffffffu, 0xffffffffu};
    for (int k = 0; k < D; ++k) {
      const uint32_t w = ecmp[(size_t)k * N + i];
      if (w != 0u) {
        const int ob = (int)(int16_t)(w & 0xffffu), oc = (int)w >> 16;
        int jb = 0, jc = 0;
        while (o[jb] != ob) ++jb;
        while (o[jc] != oc) ++jc;
        const int sh = 8 * (k & 3);
        mw[k >> 2] = (mw[k >> 2] & ~(0xffu << sh)) | ((uint32_t)(jb | (jc << 4)) << sh);
      }
    }
    nmap[i] = make_uint2(mw[0], mw[1]);
  }
  if (maxcnt) {
    most = __reduce_max_sync(0xffffffffu, most);
    if ((threadIdx.x & 31) == 0) atomicMax(maxcnt, most);
  }
}

// A row's merged coefficients, accumulated entry by entry in incidence-slot
// order (b before c within an entry), then stored: the same order whichever
// schedule produced the entries.
template <typename R> struct NbAcc {
  R a[kNbMax];
  uint2 map;  // the row's slot map
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int j = 0; j < kNbMax; ++j) a[j] = R(0);
    map = make_uint2(0xffffffffu, 0xffffffffu);
  }
  __device__ __forceinline__ void load_map(const Params<R> &P, int i) { map = __ldg(&P.nmap[i]); }
  __device__ __forceinline__ void add(int k, typename Params<R>::R2 c) {
    const unsigned m = ((k < 4 ? map.x : map.y) >> (8 * (k & 3))) & 0xffu;
    if (m == 0xffu) return;
    const unsigned jb = m & 15u, jc = m >> 4;
#pragma unroll
    for (int j = 0; j < kNbMax; ++j) {
      if (jb == (unsigned)j) a[j] = radd(a[j], c.x);
      if (jc == (unsigned)j) a[j] = radd(a[j], c.y);
    }
  }
  __device__ __forceinline__ void store(const Params<R> &P, int i) const {
#pragma unroll
    for (int j = 0; j < kNbMax; ++j)
      if (j < P.Dn) P.nbc[(size_t)j * P.N + i] = a[j];
  }
};

// Whether a right-hand-side pass merges rows (merged rows present; the
// staged families' passes run without records).
template <typename R>
__device__ __forceinline__ bool nb_merging(const Params<R> &P) {
  return P.nbc != nullptr;
}

// Coefficients kappa_e A_e and mA = c_e A_e / 12 of element e's damage
// operator (c_e = cbase + 2 H_e, both scaled by the toughness field), with
// every rounding spelled out so that each caller gets the same bits.
template <typename R>
__device__ __forceinline__ void dmg_coefs(const Params<R> &P, int e, R A, R h, R sg, R &kA, R &mA) {
  const R c = rfma(P.cbase, sg, R(2) * h);
  kA = rmul(rmul(P.kappa, sg), A);
  mA = rmul(rmul(c, A), R(1) / R(12));
}

// Row i's merged coefficients with its entries' coefficients evaluated
// again here (the entry-parallel schedule, whose entries are evaluated by
// other threads of the block): rhs_entry's arithmetic.
template <typename R>
__device__ __forceinline__ void nb_merge_row(const Params<R> &P, int i) {
  if (!nb_merging(P)) return;
  typedef typename Params<R>::R4 R4;
  NbAcc<R> acc;
  acc.zero();
  acc.load_map(P, i);
  for (int k = 0; k < P.D; ++k) {
    const int en = __ldg(&P.ell[(size_t)k * P.N + i]);
    if (en < 0) continue;
    const int e = en >> 2;
    int4 t;
    R A;
    R4 G;
    load_elem(P, e, t, A, G);
    R kA, mA;
    dmg_coefs(P, e, A, P.Hr[e], gc_scale(P, e), kA, mA);
    acc.add(k, erec_coef<R>(G, en & 3, kA, mA));
  }
  acc.store(P, i);
}

// Row i of the merged operator applied to the values val(j) of its
// neighbours, added to q (diag_i times the row's own value): all DN
// records, then all DN neighbour gathers in flight, then an explicit fma
// chain in slot order (padding slots add an exact 0).
template <int DN, typename R, typename F>
__device__ __forceinline__ R nb_row(const Params<R> &P, int i, R q, F val) {
  uint32_t w[DN / 2];
  R c[DN], v[DN];
#pragma unroll
  for (int j = 0; j < DN / 2; ++j) w[j] = __ldg(&P.nbo[(size_t)j * P.N + i]);
#pragma unroll
  for (int j = 0; j < DN; ++j) c[j] = __ldg(&P.nbc[(size_t)j * P.N + i]);
#pragma unroll
  for (int j = 0; j < DN; ++j) {
    const uint32_t x = w[j >> 1];
    const int o = (j & 1) ? (int)x >> 16 : (int)(int16_t)(x & 0xffffu);
    v[j] = val(i + o);
  }
#pragma unroll
  for (int j = 0; j < DN; ++j) q = fma(c[j], v[j], q);
  return q;
}

template <typename R, typename F>
__device__ __forceinline__ R nb_row_any(const Params<R> &P, int i, R q, F val) {
  return P.Dn <= 6 ? nb_row<6>(P, i, q, val) : nb_row<8>(P, i, q, val);
}

// The damage record of an element from its geometry and coefficients.
template <typename R>
__device__ __forceinline__ DRec<R> make_drec(const int4 &t, const typename Params<R>::R4 &G, R kA, R mA) {
  const R g2x = -(G.x + G.z), g2y = -(G.y + G.w);
  DRec<R> o;
  o.n0 = t.x;
  o.n1 = t.y;
  o.n2 = t.z;
  o.w01 = kA * (G.x * G.z + G.y * G.w);
  o.w02 = kA * (G.x * g2x + G.y * g2y);
  o.w12 = kA * (G.z * g2x + G.w * g2y);
  o.mA = mA;
  return o;
}

template <typename R>
__device__ __forceinline__ void load_drec(const Params<R> &P, int e, int &n0, int &n1, int &n2, R &w01, R &w02,
                                          R &w12, R &mA) {
  const DRec<R> *rp = P.drec + e;
  if constexpr (sizeof(R) == 4) {
    unsigned v0, v1, v2, v3, v4, v5, v6, v7;
    asm("ld.global.nc.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=r"(v0), "=r"(v1), "=r"(v2), "=r"(v3), "=r"(v4), "=r"(v5), "=r"(v6), "=r"(v7)
        : "l"(rp));
    (void)v7;
    n0 = (int)v0;
    n1 = (int)v1;
    n2 = (int)v2;
    w01 = __uint_as_float(v3);
    w02 = __uint_as_float(v4);
    w12 = __uint_as_float(v5);
    mA = __uint_as_float(v6);
  } else {
    const int4 n = __ldg(reinterpret_cast<const int4 *>(rp));
    const double2 a = __ldg(reinterpret_cast<const double2 *>(rp) + 1);
    const double2 b = __ldg(reinterpret_cast<const double2 *>(rp) + 2);
    n0 = n.x;
    n1 = n.y;
    n2 = n.z;
    w01 = (R)a.x;
    w02 = (R)a.y;
    w12 = (R)b.x;
    mA = (R)b.y;
  }
}

// Damage records of every element from the geometry and the history P.Hr
// (element-parallel; the forward's right-hand-side kernels write them as a
// by-product instead).
template <typename R>
__global__ void __launch_bounds__(256) k_drec_build(Params<R> P) {
  typedef typename Params<R>::R4 R4;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < P.Ne; e += gridDim.x * blockDim.x) {
    int4 t;
    R A;
    R4 G;
    load_elem(P, e, t, A, G);
    const R sg = gc_scale(P, e);
    const R kA = (P.kappa * sg) * A;
    const R mA = (P.cbase * sg + R(2) * P.Hr[e]) * A * (R(1) / R(12));
    P.drec[e] = make_drec<R>(t, G, kA, mA);
  }
}

// Right-hand side, Jacobi diagonal and lifted initial residual of the
// damage problem (AT2: Eq. damage_pde_at2; AT1: Eq. damage_pde_at1), one
// incidence entry's share: (b, diag, (A x0)_a, (A 1_D)_a) with
// x0 = d_prev (1 on the notch).
// With cf, a merging pass's entry coefficients are returned there instead
// of written to the entry records.
// rhs_entry's arithmetic on an element already loaded (t, A, G), its
// history h in the kernel precision and toughness scale sg (the fused
// force and right-hand-side kernel calls this directly).
// The entry's four terms from its element's load density w, coefficients
// kA, mA, the notch flags n0..n2 and x0 = d_prev of its three nodes.
template <typename R>
__device__ __forceinline__ typename Params<R>::R4 rhs_entry_terms(int a, R A, const typename Params<R>::R4 &G, R w,
                                                                  R kA, R mA, bool n0, bool n1, bool n2, R x0, R x1,
                                                                  R x2) {
  typedef typename Params<R>::R4 R4;
  R gx, gy;
  slot_grad<R>(G, a, gx, gy);
  R4 o;
  o.x = rmul(rmul(w, A), R(1) / R(3));
  o.y = rfma(kA, rfma(gx, gx, rmul(gy, gy)), rmul(R(2), mA));
  o.z = elem_row<R>(G, a, kA, mA, x0, x1, x2);
  o.w = (n0 || n1 || n2) ? elem_row<R>(G, a, kA, mA, n0 ? R(1) : R(0), n1 ? R(1) : R(0), n2 ? R(1) : R(0))
                         : R(0);
  return o;
}

template <typename R>
__device__ __forceinline__ typename Params<R>::R4 rhs_entry_core(const Params<R> &P, int e, int a, const int4 &t,
                                                                 R A, const typename Params<R>::R4 &G, R h, R sg,
                                                                 int slot, int node, int csr,
                                                                 typename Params<R>::R2 *cf, uint32_t fm = kFanLoad) {
  typedef typename Params<R>::R4 R4;
  const R w = rfma(P.wbase, sg, rmul(R(2), h));
  const bool n0 = P.flags[t.x] & kNotch, n1 = P.flags[t.y] & kNotch, n2 = P.flags[t.z] & kNotch;
  const R x0 = n0 ? R(1) : P.dprev[t.x];
  const R x1 = n1 ? R(1) : P.dprev[t.y];
  const R x2 = n2 ? R(1) : P.dprev[t.z];
  R kA, mA;
  dmg_coefs(P, e, A, h, sg, kA, mA);
  if (a == 0 && P.drec) P.drec[e] = make_drec<R>(t, G, kA, mA);
  if (cf) {
    *cf = erec_coef<R>(G, a, kA, mA);
  } else if (has_erec(P)) {
    // the entry's incidence slot: given, or from its CSR position
    if (slot < 0 && csr >= 0) {
      node = a == 0 ? t.x : (a == 1 ? t.y : t.z);
      slot = csr - __ldg(&P.ptr[node]);
    }
    if (slot >= 0) put_erec(P, slot, node, G, a, kA, mA, fm);
  }
  return rhs_entry_terms<R>(a, A, G, w, kA, mA, n0, n1, n2, x0, x1, x2);
}

template <typename R>
__device__ __forceinline__ typename Params<R>::R4 rhs_entry(const Params<R> &P, int en, int slot = -1,
                                                            int node = -1, int csr = -1,
                                                            typename Params<R>::R2 *cf = nullptr,
                                                            uint32_t fm = kFanLoad) {
  typedef typename Params<R>::R4 R4;
  const int e = en >> 2, a = en & 3;
  int4 t;
  R A;
  R4 G;
  load_elem(P, e, t, A, G);
  return rhs_entry_core<R>(P, e, a, t, A, G, P.Hr[e], gc_scale(P, e), slot, node, csr, cf, fm);
}

// Node i of the right-hand side: r = b - A x0, b_eff = b - A 1_D, the
// Jacobi inverse diagonal and z = r / diag; accumulates |b_eff|^2, |r|^2
// and r.z.
template <typename R>
__device__ __forceinline__ void rhs_node(const Params<R> &P, int i, R bi, R dg, R ax, R a1,
                                         typename Acc<R>::T (&vals)[3]) {
  typedef Acc<R> AC;
  const R ri = bi - ax, be = bi - a1;
  const R di = R(1) / dg;
  if (P.diag) P.diag[i] = dg;
  const R zi = ri * di;
  P.x[i] = P.dprev[i];
  P.r[i] = ri;
  P.dinv[i] = di;
  typename Params<R>::R2 pz;
  pz.x = R(0);
  pz.y = zi;
  P.pz[i] = pz;
  if (P.b) P.b[i] = bi;
  const R sr = P.rscale * ri, sb = P.rscale * be;
  vals[0] = AC::add(vals[0], AC::prod(sb, sb));
  vals[1] = AC::add(vals[1], AC::prod(sr, sr));
  vals[2] = AC::add(vals[2], AC::prod(sr, zi));
}

template <typename R>
__device__ __forceinline__ void rhs_notch_node(const Params<R> &P, int i) {
  P.x[i] = R(1);
  P.r[i] = R(0);
  typename Params<R>::R2 pz;
  pz.x = R(0);
  pz.y = R(0);
  P.pz[i] = pz;
  P.dinv[i] = R(0);
  if (P.b) P.b[i] = R(0);
}

// Last block of the right-hand side: solve scalars and the loop condition.
template <typename R>
__device__ __forceinline__ void rhs_finish(const Params<R> &P, const double *tot) {
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
  const bool done = (P.model == kAT2) && (S.bn == 0.0 || sqrt(S.rr) <= P.tol * S.bn);
  S.done = done ? 1 : 0;
  if (P.use_cond) cudaGraphSetConditional(P.cond_inner, done ? 0u : 1u);
}

template <typename R>
__global__ void __launch_bounds__(256) k_dmg_rhs_ep(Params<R> P) {
  typedef typename Params<R>::R4 R4;
  typedef Acc<R> AC;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R4 *cc = reinterpret_cast<R4 *>(smem_raw);
  typename AC::T vals[3] = {AC::zero(), AC::zero(), AC::zero()};
  for (int b = blockIdx.x; b < P.nblk; b += gridDim.x) {
    int i0, i1, k0, k1;
    block_nodes(P, b, i0, i1, k0, k1);
    for (int k = k0 + threadIdx.x; k < k1; k += blockDim.x) cc[k - k0] = rhs_entry(P, __ldg(&P.ent[k]), -1, -1, k);
    __syncthreads();
    for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
      if (P.flags[i] & kNotch) {
        rhs_notch_node(P, i);
        continue;
      }
      const int j0 = __ldg(&P.ptr[i]) - k0, j1 = __ldg(&P.ptr[i + 1]) - k0;
      R bi = 0, dg = 0, ax = 0, a1 = 0;
      for (int j = j0; j < j1; ++j) {
        const R4 o = cc[j];
        bi = radd(bi, o.x);
        dg = radd(dg, o.y);
        ax = radd(ax, o.z);
        a1 = radd(a1, o.w);
      }
      rhs_node(P, i, bi, dg, ax, a1, vals);
      nb_merge_row(P, i);
    }
    __syncthreads();
  }
  __shared__ double tot[3];
  if (reduce_last<R, 3>(vals, P.part, P.ticket, tot) && threadIdx.x == 0) rhs_finish(P, tot);
}

// A notch node has no row, but the elements it holds in slot 0 still need
// their damage records (written by rhs_entry as a by-product).
template <typename R>
__device__ __forceinline__ void drec_notch_node(const Params<R> &P, int i) {
  if (!P.drec) return;
  for (int k = 0; k < P.D; ++k) {
    const int en = __ldg(&P.ell[(size_t)k * P.N + i]);
    if (en >= 0 && (en & 3) == 0) (void)rhs_entry(P, en);
  }
}

// FP32: four CTAs per SM (at most 64 registers; the U > 1 variants spill a
// little, measured faster than three CTAs without spills).
template <typename R, int U>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 4 : 1) k_dmg_rhs_nc(Params<R> P) {
  typedef typename Params<R>::R4 R4;
  typedef Acc<R> AC;
  typename AC::T vals[3] = {AC::zero(), AC::zero(), AC::zero()};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.N; i += gridDim.x * blockDim.x) {
    if (P.flags[i] & kNotch) {
      rhs_notch_node(P, i);
      drec_notch_node(P, i);
      continue;
    }
    R bi = 0, dg = 0, ax = 0, a1 = 0;
    const bool merge = nb_merging(P);
    NbAcc<R> nacc;
    nacc.zero();
    if (merge) nacc.load_map(P, i);
    const uint32_t fm = fan_word(P, i);
    for (int k = 0; k < P.D; k += U) {
      R4 o[U];
      typename Params<R>::R2 cf[U];
      int en[U];
#pragma unroll
      for (int u = 0; u < U; ++u) en[u] = k + u < P.D ? __ldg(&P.ell[(size_t)(k + u) * P.N + i]) : -1;
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (en[u] >= 0) o[u] = rhs_entry(P, en[u], k + u, i, -1, merge ? &cf[u] : nullptr, fm);
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
    rhs_node(P, i, bi, dg, ax, a1, vals);
    if (merge) nacc.store(P, i);
  }
  __shared__ double tot[3];
  if (reduce_last<R, 3>(vals, P.part, P.ticket, tot) && threadIdx.x == 0) rhs_finish(P, tot);
}

// Force and damage right-hand side in one pass (node-centric, U entries in
// flight): per incidence entry the element's strain, split, degraded stress
// and psi+ (force_entry's arithmetic), the history H_{n+1} = max(H_n, psi+)
// that the entry's element will hold after this pass, and the damage
// right-hand side's terms from that history (rhs_entry's arithmetic on the
// element already loaded); per node the corrector and the solve's set-up
// (rhs_node), per block the reductions of the set-up.  Results are those
// of the force kernel followed by the right-hand-side kernel: the history
// each thread uses is max(H_n, psi+) taken the way history_update takes it,
// whether or not the element's owner entry has already stored it (max is
// idempotent), so no thread depends on another's write.  FP32: four CTAs
// per SM (64 registers: U = 1 fits without spills; 109 against 124 us for
// three CTAs on the 1M-node plate).
template <typename R>
__device__ __forceinline__ void force_rhs_entry(const Params<R> &P, int en, int slot, int node, R &fx, R &fy, R &psip,
                                                typename Params<R>::R4 &o, typename Params<R>::R2 *cf, uint32_t fm) {
  typedef typename Params<R>::R4 R4;
  const int e = en >> 2, a = en & 3;
  int4 t;
  R A;
  R4 G;
  load_elem(P, e, t, A, G);
  R exx, eyy, exy;
  elem_strain(P, G, t, exx, eyy, exy);
  const R db = rmul(radd(radd(P.d[t.x], P.d[t.y]), P.d[t.z]), R(1) / R(3));
  const R g = rfma(R(1) - db, R(1) - db, P.eta);
  R sxx, syy, sxy;
  stress(P, exx, eyy, exy, g, sxx, syy, sxy, psip);
  R gx, gy;
  slot_grad<R>(G, a, gx, gy);
  slot_force(A, sxx, syy, sxy, gx, gy, fx, fy);
  R h;
  if constexpr (sizeof(R) == 8) {
    const double ho = P.H[e], hp = (double)psip;
    h = hp > ho ? hp : ho;
  } else {
    const long long pb = f2d_bits((float)psip);
    const long long hb = __double_as_longlong(P.H[e]);
    h = pb > hb ? (float)psip : (float)__longlong_as_double(hb);
  }
  o = rhs_entry_core<R>(P, e, a, t, A, G, h, gc_scale(P, e), slot, node, -1, cf, fm);
}

template <typename R, int U>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 4 : 1) k_force_rhs_nc(Params<R> P) {
  typedef typename Params<R>::R4 R4;
  typedef Acc<R> AC;
  typename AC::T vals[3] = {AC::zero(), AC::zero(), AC::zero()};
  const double S = load_scale(P, 1);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.N; i += gridDim.x * blockDim.x) {
    const bool notch = P.flags[i] & kNotch;
    const bool merge = !notch && nb_merging(P);
    R fx = 0, fy = 0, bi = 0, dg = 0, ax = 0, a1 = 0;
    NbAcc<R> nacc;
    nacc.zero();
    if (merge) nacc.load_map(P, i);
    const uint32_t fm = fan_word(P, i);
    for (int k = 0; k < P.D; k += U) {
      int en[U];
      R cx[U], cy[U], pp[U];
      R4 o[U];
      typename Params<R>::R2 cf[U];
#pragma unroll
      for (int u = 0; u < U; ++u) en[u] = k + u < P.D ? __ldg(&P.ell[(size_t)(k + u) * P.N + i]) : -1;
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (en[u] >= 0)  // a notch row has no damage row: only the element records are written
          force_rhs_entry(P, en[u], notch ? -1 : k + u, i, cx[u], cy[u], pp[u], o[u], merge ? &cf[u] : nullptr, fm);
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (en[u] >= 0) {
          fx = radd(fx, cx[u]);
          fy = radd(fy, cy[u]);
          history_update(P, en[u], pp[u]);
          bi = radd(bi, o[u].x);
          dg = radd(dg, o[u].y);
          ax = radd(ax, o[u].z);
          a1 = radd(a1, o[u].w);
          if (merge) nacc.add(k + u, cf[u]);
        }
    }
    corrector(P, i, fx, fy, S);
    if (notch) {
      rhs_notch_node(P, i);
    } else {
      rhs_node(P, i, bi, dg, ax, a1, vals);
      if (merge) nacc.store(P, i);
    }
  }
  __shared__ double tot[3];
  if (reduce_last<R, 3>(vals, P.part, P.ticket, tot) && threadIdx.x == 0) rhs_finish(P, tot);
}

// Next search direction at node j: p_new = z + beta p_old (zero on the
// notch and, for AT1, outside the free set).  The same expression is
// evaluated by the matvec (for neighbours) and the update (for the node).
template <typename R>
__device__ __forceinline__ R pnew(const Params<R> &P, int j, R beta) {
  const typename Params<R>::R2 v = P.pz[j];
  return fma(beta, v.x, v.y);
}

// Fan rows: the row's six distinct-neighbour values val(i + o) gathered
// once, then per fan position k the triangle's two coefficients applied to
// v_k and v_{k+1 mod m} (explicit fma and non-contracted adds, positions in
// order; positions past the fan have zero coefficients and add an exact 0).
// fan_row_w takes the row's fan words w and fan length m already loaded;
// fan_sum is the row's sum once coefficients and neighbour values are in
// registers.
__device__ __forceinline__ int fan_offset(const uint32_t (&w)[3], int j) {
  const uint32_t x = w[j >> 1];
  return (j & 1) ? (int)x >> 16 : (int)(int16_t)(x & 0xffffu);
}

template <typename R, typename C2>
__device__ __forceinline__ R fan_sum(R q, const C2 (&cf)[6], const R (&v)[6], int m) {
  R c[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const R vc = (k + 1 == m) ? v[0] : v[k < 5 ? k + 1 : 0];
    c[k] = rfma(cf[k].x, v[k], rmul(cf[k].y, vc));
  }
#pragma unroll
  for (int k = 0; k < 6; ++k) q = radd(q, c[k]);
  return q;
}

template <typename R, typename C2, typename F>
__device__ __forceinline__ R fan_row_w(const Params<R> &P, const C2 *cfs, int i, R q, const uint32_t (&w)[3], int m,
                                       F val) {
  C2 cf[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    if (k < P.D) {
      cf[k] = __ldg(&cfs[(size_t)k * P.N + i]);
    } else {
      cf[k].x = 0;
      cf[k].y = 0;
    }
  }
  R v[6];
#pragma unroll
  for (int j = 0; j < 6; ++j) v[j] = val(i + fan_offset(w, j));
  return fan_sum(q, cf, v, m);
}

template <typename R, typename C2, typename F>
__device__ __forceinline__ R fan_row(const Params<R> &P, const C2 *cfs, int i, R q, F val) {
  uint32_t w[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) w[j] = __ldg(&P.fno[(size_t)j * P.N + i]);
  return fan_row_w(P, cfs, i, q, w, (int)(__ldg(&P.fmap[i]) >> 24), val);
}

// Row i of q = A p_new from the FP32 entry records: diag_i p_i, then per
// incidence slot in order (U records in flight) c_b p_b + c_c p_c, rounded
// the same way in every schedule (explicit fma and non-contracted adds).
// Compact records add an exact 0 for empty slots.
template <int U>
__device__ __forceinline__ float erec_row(const Params<float> &P, int i, float beta, float pc) {
  float q = P.diag[i] * pc;
  if (P.nbc) return nb_row_any(P, i, q, [&](int j) { return pnew(P, j, beta); });
  if (P.fno) return fan_row(P, P.ecf, i, q, [&](int j) { return pnew(P, j, beta); });
  if (P.ecmp) {
    if (U >= 3 && P.D <= 6) {
      // the whole row at once: six slots' records, then their twelve
      // neighbour gathers in flight together (slots past D add an exact 0)
      uint32_t w[6];
      float2 cf[6];
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        const bool in = k < P.D;
        w[k] = in ? __ldg(&P.ecmp[(size_t)k * P.N + i]) : 0u;
        cf[k] = in ? __ldg(&P.ecf[(size_t)k * P.N + i]) : make_float2(0.f, 0.f);
      }
      float c[6];
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        const int ob = (int)(int16_t)(w[k] & 0xffffu), oc = (int)w[k] >> 16;
        c[k] = fmaf(cf[k].x, pnew(P, i + ob, beta), __fmul_rn(cf[k].y, pnew(P, i + oc, beta)));
      }
#pragma unroll
      for (int k = 0; k < 6; ++k) q = __fadd_rn(q, c[k]);
      return q;
    }
    for (int k = 0; k < P.D; k += U) {
      uint32_t w[U];
      float2 cf[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const bool in = k + u < P.D;
        w[u] = in ? __ldg(&P.ecmp[(size_t)(k + u) * P.N + i]) : 0u;
        cf[u] = in ? __ldg(&P.ecf[(size_t)(k + u) * P.N + i]) : make_float2(0.f, 0.f);
      }
      float c[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int ob = (int)(int16_t)(w[u] & 0xffffu), oc = (int)w[u] >> 16;
        c[u] = fmaf(cf[u].x, pnew(P, i + ob, beta), __fmul_rn(cf[u].y, pnew(P, i + oc, beta)));
      }
#pragma unroll
      for (int u = 0; u < U; ++u) q = __fadd_rn(q, c[u]);
    }
    return q;
  }
  for (int k = 0; k < P.D; k += U) {
    float4 er[U];
#pragma unroll
    for (int u = 0; u < U; ++u)
      er[u] = k + u < P.D ? __ldg(&P.erec[(size_t)(k + u) * P.N + i]) : make_float4(__int_as_float(-1), 0.f, 0.f, 0.f);
    float c[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int nb = __float_as_int(er[u].x);
      if (nb >= 0) c[u] = fmaf(er[u].z, pnew(P, nb, beta), __fmul_rn(er[u].w, pnew(P, __float_as_int(er[u].y), beta)));
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (__float_as_int(er[u].x) >= 0) q = __fadd_rn(q, c[u]);
  }
  return q;
}

// Element-wise rows with shared gathers: a row's six entry records (two
// element coefficients each, Eq. matrix_free_fe_operator applied element
// by element) use the values of the row's distinct neighbours, each
// gathered once, picked per entry through the slot map.  The arithmetic is
// erec_row's whole-row form term for term (c_b p_b + c_c p_c per entry,
// then summed in slot order; an empty slot uses the row's own value with
// zero coefficients), so the result is bit-identical to it: only loads are
// shared, no two elements' coefficients are combined.
struct ElRow6 {
  uint32_t w[3];  // the row's distinct neighbour offsets, two per word
  uint2 map;      // incidence slot k -> (jb | jc << 4), 0xff = empty
  float2 cf[6];   // entry k's element coefficients of p_b and p_c
  float dg;       // Jacobi diagonal
  unsigned fl;
};

__device__ __forceinline__ void el_load6(const Params<float> &P, int i, ElRow6 &r) {
#pragma unroll
  for (int j = 0; j < 3; ++j) r.w[j] = __ldg(&P.gnbo[(size_t)j * P.N + i]);
  r.map = __ldg(&P.gmap[i]);
#pragma unroll
  for (int k = 0; k < 6; ++k)
    r.cf[k] = k < P.D ? __ldg(&P.ecf[(size_t)k * P.N + i]) : make_float2(0.f, 0.f);
  r.dg = __ldg(&P.diag[i]);
  r.fl = __ldg(&P.flags[i]);
}

// Value of merged slot j among the gathered v[0..5]; any other j (the
// empty-slot code 15) gives the row's own value self.
__device__ __forceinline__ float el_pick(const float (&v)[6], unsigned j, float self) {
  float r = self;
#pragma unroll
  for (int t = 0; t < 6; ++t) r = j == (unsigned)t ? v[t] : r;
  return r;
}

// q (= diag p_i) plus the row's entries applied to the gathered values.
__device__ __forceinline__ float el_apply6(const ElRow6 &r, const float (&v)[6], float self, float q) {
  float c[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const unsigned m = ((k < 4 ? r.map.x : r.map.y) >> (8 * (k & 3))) & 0xffu;
    const float vb = el_pick(v, m & 15u, self), vc = el_pick(v, m >> 4, self);
    c[k] = fmaf(r.cf[k].x, vb, __fmul_rn(r.cf[k].y, vc));
  }
#pragma unroll
  for (int k = 0; k < 6; ++k) q = __fadd_rn(q, c[k]);
  return q;
}

template <typename F>
__device__ __forceinline__ void el_gather6(const ElRow6 &r, int i, float (&v)[6], F val) {
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    const uint32_t x = r.w[j >> 1];
    const int o = (j & 1) ? (int)x >> 16 : (int)(int16_t)(x & 0xffffu);
    v[j] = val(i + o);
  }
}

// Row i of q = A p_new from the FP64 entry records: erec_row's arithmetic
// in FP64 (diag_i p_i, then per incidence slot c_b p_b + c_c p_c, U slots
// in flight, summed in slot order; empty slots add an exact 0).
template <int U>
__device__ __forceinline__ double erec_row_d(const Params<double> &P, int i, double beta, double pc) {
  double q = P.diag[i] * pc;
  if (P.fno) return fan_row(P, P.ecfd, i, q, [&](int j) { return pnew(P, j, beta); });
  for (int k = 0; k < P.D; k += U) {
    uint32_t w[U];
    double2 cf[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const bool in = k + u < P.D;
      w[u] = in ? __ldg(&P.ecmp[(size_t)(k + u) * P.N + i]) : 0u;
      cf[u] = in ? __ldg(&P.ecfd[(size_t)(k + u) * P.N + i]) : make_double2(0.0, 0.0);
    }
    double c[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int ob = (int)(int16_t)(w[u] & 0xffffu), oc = (int)w[u] >> 16;
      c[u] = fma(cf[u].x, pnew(P, i + ob, beta), __dmul_rn(cf[u].y, pnew(P, i + oc, beta)));
    }
#pragma unroll
    for (int u = 0; u < U; ++u) q = __dadd_rn(q, c[u]);
  }
  return q;
}

// One incidence entry's share of (A p_new)_a, matrix-free (Eq.
// matrix_free_fe_operator): element coefficients are rebuilt from the
// geometry and the history on every application.
template <typename R>
__device__ __forceinline__ R mv_entry_vals(const Params<R> &P, const int4 &t, R A, const typename Params<R>::R4 &G,
                                           R h, R sg, int a, R beta, R pc) {
  const R kA = (P.kappa * sg) * A;
  const R mA = (P.cbase * sg + R(2) * h) * A * (R(1) / R(12));
  // the entry's own node (slot a) is the row's node: its value is pc
  const R p0 = a == 0 ? pc : pnew(P, t.x, beta);
  const R p1 = a == 1 ? pc : pnew(P, t.y, beta);
  const R p2 = a == 2 ? pc : pnew(P, t.z, beta);
  return elem_row<R>(G, a, kA, mA, p0, p1, p2);
}

template <typename R>
__device__ __forceinline__ R mv_entry(const Params<R> &P, int en, R beta, R pc) {
  typedef typename Params<R>::R4 R4;
  const int e = en >> 2, a = en & 3;
  if (P.drec) {
    // row a of the element operator from the solve's record: the other two
    // slots b, c and their weights w_ab, w_ac
    int n0, n1, n2;
    R w01, w02, w12, mA;
    load_drec(P, e, n0, n1, n2, w01, w02, w12, mA);
    const int nb = a == 0 ? n1 : n0, nc = a == 2 ? n1 : n2;
    const R wb = a == 2 ? w02 : w01, wc = a == 0 ? w02 : w12;
    const R pb = pnew(P, nb, beta), pcc = pnew(P, nc, beta);
    return wb * (pb - pc) + wc * (pcc - pc) + mA * (R(2) * pc + pb + pcc);
  }
  int4 t;
  R A;
  R4 G;
  load_elem(P, e, t, A, G);
  return mv_entry_vals<R>(P, t, A, G, P.Hr[e], gc_scale(P, e), a, beta, pc);
}

// Rows n0 + threadIdx.x, ... < n1 of q = A p_new from the element records
// and history staged in shared memory (srec: 32-byte records as float4
// pairs, sh: H), U entries in flight; same per-entry arithmetic and
// summation order as matvec_rows.
template <int U>
__device__ __forceinline__ void matvec_rows_staged(const Params<float> &P, float beta, int n0, int n1,
                                                   const float4 *srec, const float *sh, DF &acc) {
  typedef Acc<float> AC;
  for (int i = n0 + (int)threadIdx.x; i < n1; i += blockDim.x) {
    float q = 0.f;
    if (!is_fixed(P, i)) {
      const float pc = pnew(P, i, beta);
      for (int k = 0; k < P.D; k += U) {
        float c[U];
        unsigned sl[U];
#pragma unroll
        for (int u = 0; u < U; ++u) sl[u] = k + u < P.D ? (unsigned)P.st_slot[(size_t)(k + u) * P.st_ns + i] : 0xffffu;
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (sl[u] != 0xffffu) {
            const int sidx = (int)(sl[u] >> 2);
            const float4 r0 = srec[2 * sidx], r1 = srec[2 * sidx + 1];
            const int4 t = make_int4(__float_as_int(r0.x), __float_as_int(r0.y), __float_as_int(r0.z), 0);
            c[u] = mv_entry_vals<float>(P, t, r0.w, r1, sh[sidx], 1.f, (int)(sl[u] & 3u), beta, pc);
          }
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (sl[u] != 0xffffu) q = radd(q, c[u]);
      }
      acc = AC::add(acc, AC::prod(pnew(P, i, beta), P.rscale * q));
    }
    P.q[i] = q;
  }
}

template <typename R>
__device__ __forceinline__ void matvec_finish(const Params<R> &P, const double *tot) {
  SolveScalars &S = *P.sc;
  S.pq = tot[0];
  S.alpha = tot[0] != 0.0 ? S.rho / tot[0] : 0.0;
  S.alpha_f = (float)S.alpha;
}

// q = A p_new on free rows and the reduction p_new . q -> alpha = rho/(p.q).
// Entry-parallel schedule.
template <typename R>
__global__ void __launch_bounds__(256) k_cg_matvec_ep(Params<R> P) {
  typedef Acc<R> AC;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R *cq = reinterpret_cast<R *>(smem_raw);
  typename AC::T vals[1] = {AC::zero()};
  const R beta = sc_beta<R>(P.sc);
  if (P.nbc || has_erec(P)) {
    {
      // merged rows or FP32 entry records: rows of the block's nodes, the
      // same per-row arithmetic as the node-centric schedules
      for (int b = blockIdx.x; b < P.nblk; b += gridDim.x) {
        const int i0 = b * P.NB, i1 = min(i0 + P.NB, P.N);
        for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
          R q = 0;
          if (!is_fixed(P, i)) {
            const R pc = pnew(P, i, beta);
            if constexpr (sizeof(R) == 4)
              q = erec_row<1>(P, i, beta, pc);
            else if (P.nbc)
              q = nb_row_any(P, i, P.diag[i] * pc, [&](int j) { return pnew(P, j, beta); });
            else
              q = erec_row_d<1>(P, i, beta, pc);
            vals[0] = AC::add(vals[0], AC::prod(pc, P.rscale * q));
          }
          P.q[i] = q;
        }
      }
      __shared__ double tot1[1];
      if (reduce_last<R, 1>(vals, P.part, P.ticket, tot1) && threadIdx.x == 0) matvec_finish(P, tot1);
      return;
    }
  }
  for (int b = blockIdx.x; b < P.nblk; b += gridDim.x) {
    int i0, i1, k0, k1;
    block_nodes(P, b, i0, i1, k0, k1);
    for (int k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
      const int en = __ldg(&P.ent[k]);
      const int e = en >> 2, a = en & 3;
      const int4 t = make_int4(P.rec[e].n0, P.rec[e].n1, P.rec[e].n2, 0);
      const int node = a == 0 ? t.x : (a == 1 ? t.y : t.z);
      cq[k - k0] = mv_entry(P, en, beta, pnew(P, node, beta));
    }
    __syncthreads();
    for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
      R q = 0;
      if (!is_fixed(P, i)) {
        const int j0 = __ldg(&P.ptr[i]) - k0, j1 = __ldg(&P.ptr[i + 1]) - k0;
        for (int j = j0; j < j1; ++j) q = radd(q, cq[j]);
        vals[0] = AC::add(vals[0], AC::prod(pnew(P, i, beta), P.rscale * q));
      }
      P.q[i] = q;
    }
    __syncthreads();
  }
  __shared__ double tot[1];
  if (reduce_last<R, 1>(vals, P.part, P.ticket, tot) && threadIdx.x == 0) matvec_finish(P, tot);
}

// One width-6 merged row's records: neighbour offsets (three words), merged
// coefficients, diagonal and flags.
struct NbRow6 {
  uint32_t w[3];
  float c[6];
  float dg;
  unsigned fl;
};

__device__ __forceinline__ void nb_load6(const Params<float> &P, int i, NbRow6 &r) {
#pragma unroll
  for (int j = 0; j < 3; ++j) r.w[j] = __ldg(&P.nbo[(size_t)j * P.N + i]);
#pragma unroll
  for (int j = 0; j < 6; ++j) r.c[j] = __ldg(&P.nbc[(size_t)j * P.N + i]);
  r.dg = __ldg(&P.diag[i]);
  r.fl = __ldg(&P.flags[i]);
}

// Width-6 merged rows i0, i0 + stride, ... of q = A p_new, software-
// pipelined: the next row's records load while this row's neighbour values
// are gathered; cur holds row i0's records.  Same arithmetic as erec_row.
__device__ __forceinline__ void nb_rows6(const Params<float> &P, float beta, int i0, int stride, DF &acc,
                                         NbRow6 cur, int n, int ifirst, bool rev) {
  typedef Acc<float> AC;
  const int step = rev ? -stride : stride;
  for (int i = ifirst; rev ? i >= i0 : i < n; i += step) {
    NbRow6 nxt;
    const int in = i + step;
    if (rev ? in >= i0 : in < n) nb_load6(P, in, nxt);
    float q = 0.f;
    if (!((cur.fl & kNotch) || (P.freef && !P.freef[i]))) {
      const float pc = pnew(P, i, beta);
      q = cur.dg * pc;
      float v[6];
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        const uint32_t x = cur.w[j >> 1];
        const int o = (j & 1) ? (int)x >> 16 : (int)(int16_t)(x & 0xffffu);
        v[j] = pnew(P, i + o, beta);
      }
#pragma unroll
      for (int j = 0; j < 6; ++j) q = fmaf(cur.c[j], v[j], q);
      acc = AC::add(acc, AC::prod(pc, P.rscale * q));
    }
    P.q[i] = q;
    cur = nxt;
  }
}

// Node-centric rows i0, i0 + stride, ... of q = A p_new (U gathers in
// flight; merged rows of width 6: U >= 2 pipelines rows) with their share of
// p_new . q added to acc.
template <typename R, int U>
__device__ __forceinline__ void matvec_rows(const Params<R> &P, R beta, int i0, int stride,
                                            typename Acc<R>::T &acc, int iend = -1, bool rev = false) {
  typedef Acc<R> AC;
  const int n = iend < 0 ? P.N : iend;  // rows i0, i0 + stride, ... below n
  // rev: the same rows, last first (the element-wise rows of the persistent
  // loop alternate directions between iterations, so that each pass starts
  // on the records and vectors the previous one touched last)
  const int ilast = i0 < n ? i0 + (n - 1 - i0) / stride * stride : i0 - stride;
  if constexpr (sizeof(R) == 8) {
    if (P.nbc || P.ecfd) {  // FP64 merged rows or entry records
      const int istep = rev ? -stride : stride;
      for (int i = rev ? ilast : i0; rev ? i >= i0 : i < n; i += istep) {
        R q = 0;
        if (!is_fixed(P, i)) {
          const R pc = pnew(P, i, beta);
          q = P.nbc ? nb_row_any(P, i, P.diag[i] * pc, [&](int j) { return pnew(P, j, beta); })
                    : erec_row_d<U>(P, i, beta, pc);
          acc = AC::add(acc, AC::prod(pc, P.rscale * q));
        }
        P.q[i] = q;
      }
      return;
    }
  }
  if constexpr (sizeof(R) == 4) {
    if (U >= 2 && P.nbc && P.Dn <= 6) {
      NbRow6 first;
      const int ifirst = rev ? ilast : i0;
      if (i0 < n) nb_load6(P, ifirst, first);
      nb_rows6(P, beta, i0, stride, acc, first, n, ifirst, rev);
      return;
    }
    if (has_erec(P)) {
      // FP32 entry records: the row's diagonal times its own value, then per
      // entry the two other nodes' values times their coefficients (the
      // records stream in coalesced; only the p gathers are indirect)
      const int istep = rev ? -stride : stride;
      for (int i = rev ? ilast : i0; rev ? i >= i0 : i < n; i += istep) {
        R q = 0;
        if (!is_fixed(P, i)) {
          const R pc = pnew(P, i, beta);
          q = erec_row<U>(P, i, beta, pc);
          acc = AC::add(acc, AC::prod(pc, P.rscale * q));
        }
        P.q[i] = q;
      }
      return;
    }
  }
  for (int i = i0; i < n; i += stride) {
    R q = 0;
    if (!is_fixed(P, i)) {
      const R pc = pnew(P, i, beta);
      for (int k = 0; k < P.D; k += U) {
        R c[U];
        int en[U];
#pragma unroll
        for (int u = 0; u < U; ++u) en[u] = k + u < P.D ? __ldg(&P.ell[(size_t)(k + u) * P.N + i]) : -1;
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (en[u] >= 0) c[u] = mv_entry(P, en[u], beta, pc);
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (en[u] >= 0) q = radd(q, c[u]);
      }
      acc = AC::add(acc, AC::prod(pnew(P, i, beta), P.rscale * q));
    }
    P.q[i] = q;
  }
}

// Node-centric schedule of the same matvec (U gathers in flight).
template <typename R, int U>
__global__ void __launch_bounds__(256) k_cg_matvec_nc(Params<R> P) {
  typedef Acc<R> AC;
  typename AC::T vals[1] = {AC::zero()};
  const R beta = sc_beta<R>(P.sc);
  matvec_rows<R, U>(P, beta, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x, vals[0]);
  __shared__ double tot[1];
  if (reduce_last<R, 1>(vals, P.part, P.ticket, tot) && threadIdx.x == 0) matvec_finish(P, tot);
}

// x += alpha p, r -= alpha q, z = r / diag, p = p_new; reductions |r|^2 and
// r.z; the last block takes the stop decision (Sec. 2.4; stop test on the
// unpreconditioned residual).  AT1 (lo = d_prev, hi = 1): values leaving
// the box are projected and flag a restart.  FP32 handles two nodes per
// thread with 8/16-byte vector accesses (workspace arrays are padded to an
// even length; padding nodes are flagged fixed).
template <typename R>
__device__ __forceinline__ void update_node(const Params<R> &P, int i, R alpha, R beta, R &x, R &r,
                                            typename Params<R>::R2 &pz, R q, R dinv,
                                            typename Acc<R>::T (&vals)[3], bool &proj) {
  typedef Acc<R> AC;
  const R pn = fma(beta, pz.x, pz.y);
  R xi = fma(alpha, pn, x);
  const R ri = fma(-alpha, q, r);
  if (P.model == kAT1) {
    const R lo = P.dprev[i];
    if (xi < lo) { xi = lo; proj = true; }
    if (xi > R(1)) { xi = R(1); proj = true; }
  }
  const R zi = ri * dinv;
  x = xi;
  r = ri;
  pz.x = pn;
  pz.y = zi;
  const R sr = P.rscale * ri;
  vals[0] = AC::add(vals[0], AC::prod(sr, sr));
  vals[1] = AC::add(vals[1], AC::prod(sr, zi));
}

template <typename R>
__device__ __forceinline__ void update_finish(const Params<R> &P, const double *tot) {
  SolveScalars &S = *P.sc;
  bool stop = false;
  if (S.pq == 0.0) {  // p = 0: nothing moved, the iterate is exact
    if (P.model == kAT2) S.done = 1;
    stop = true;
  } else {
    S.iters += 1;
    S.rr = tot[0];
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
    }
    if (!stop && S.iters >= P.max_it) {
      stop = true;
      if (P.model == kAT2) {
        S.status = kStNotConverged;
        S.done = 1;
      }
    }
    S.beta = S.rho != 0.0 ? tot[1] / S.rho : 0.0;
    S.beta_f = (float)S.beta;
    S.rho = tot[1];
  }
  S.inner_done = stop ? 1 : 0;
  if (P.use_cond) cudaGraphSetConditional(P.cond_inner, stop ? 0u : 1u);
}

// The update of rows (pairs of rows in FP32) j0, j0 + stride, ...
template <typename R>
__device__ __forceinline__ void update_rows(const Params<R> &P, R alpha, R beta, int j0, int stride,
                                            typename Acc<R>::T (&vals)[3], bool &proj, int iend = -1,
                                            bool rev = false) {
  typedef typename Params<R>::R2 R2;
  const int n = iend < 0 ? P.N : iend;  // rows below n (FP32: pairs below (n + 1) / 2)
  if constexpr (sizeof(R) == 4) {
    const int npair = (n + 1) >> 1;
    const int jlast = j0 < npair ? j0 + (npair - 1 - j0) / stride * stride : j0 - stride;
    const int jstep = rev ? -stride : stride;
    const uchar2 *__restrict__ fl2 = reinterpret_cast<const uchar2 *>(P.flags);
    float2 *__restrict__ x2 = reinterpret_cast<float2 *>(P.x);
    float2 *__restrict__ r2 = reinterpret_cast<float2 *>(P.r);
    float4 *__restrict__ pz4 = reinterpret_cast<float4 *>(P.pz);
    const float2 *__restrict__ q2 = reinterpret_cast<const float2 *>(P.q);
    const float2 *__restrict__ d2 = reinterpret_cast<const float2 *>(P.dinv);
    for (int j = rev ? jlast : j0; rev ? j >= j0 : j < npair; j += jstep) {
      const uchar2 f = fl2[j];
      float2 xv = x2[j], rv = r2[j];
      const float2 qv = q2[j], dv = d2[j];
      const float4 pv = pz4[j];
      const int i = 2 * j;
      const bool fix0 = (f.x & kNotch) || (P.freef && !P.freef[i]);
      const bool fix1 = (f.y & kNotch) || (P.freef && !P.freef[i + 1]);
      R2 pz0, pz1;
      pz0.x = pv.x; pz0.y = pv.y;
      pz1.x = pv.z; pz1.y = pv.w;
      if (!fix0) update_node(P, i, alpha, beta, xv.x, rv.x, pz0, qv.x, dv.x, vals, proj);
      if (!fix1) update_node(P, i + 1, alpha, beta, xv.y, rv.y, pz1, qv.y, dv.y, vals, proj);
      x2[j] = xv;
      r2[j] = rv;
      pz4[j] = make_float4(pz0.x, pz0.y, pz1.x, pz1.y);
    }
  } else {
    const int ilast = j0 < n ? j0 + (n - 1 - j0) / stride * stride : j0 - stride;
    const int istep = rev ? -stride : stride;
    for (int i = rev ? ilast : j0; rev ? i >= j0 : i < n; i += istep) {
      if (is_fixed(P, i)) continue;
      R2 pz = P.pz[i];
      R x = P.x[i], r = P.r[i];
      update_node(P, i, alpha, beta, x, r, pz, P.q[i], P.dinv[i], vals, proj);
      P.x[i] = x;
      P.r[i] = r;
      P.pz[i] = pz;
    }
  }
}

template <typename R>
__global__ void __launch_bounds__(256) k_cg_update(Params<R> P) {
  typedef Acc<R> AC;
  typename AC::T vals[3] = {AC::zero(), AC::zero(), AC::zero()};
  const R beta = sc_beta<R>(P.sc);
  const R alpha = sc_alpha<R>(P.sc);
  bool proj = false;
  update_rows<R>(P, alpha, beta, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x, vals, proj);
  if (proj) vals[2] = AC::one();
  __shared__ double tot[3];
  if (reduce_last<R, 3>(vals, P.part, P.ticket, tot) && threadIdx.x == 0) update_finish(P, tot);
}

// ------------------------------------------------- persistent CG (AT2)
//
// The whole Jacobi-PCG loop of one AT2 solve in one cooperative launch
// (kPersMinBlocks CTAs of pers_threads(U, ST) per SM): per iteration the matvec
// rows, a grid all-reduce of p.q, the update rows, a grid all-reduce of
// (|r|^2, r.z).  Each all-reduce is a grid barrier: every CTA publishes its
// partial, counts itself in on S.bar with a release reduction (monotonic
// within the solve; the set-up kernel zeroes it), waits for the count with
// acquire loads, and then sums all partials itself in CTA order, so every
// CTA takes the same decisions from bit-identical totals and no second
// round trip is needed to broadcast them.  The per-row arithmetic is that
// of the kernel-per-phase loop (matvec_rows / update_rows); only the
// grouping of the partial sums differs.  Waits are bounded: after
// kSpinTimeoutNs a CTA raises S.abort, every CTA leaves, and the solve
// reports kStTimeout.

// CTA shape: two CTAs per SM; 768 threads (at most 42 registers) for one
// gather group in flight and for the staged kernels, 512 (at most 64) for
// the global-operator kernels with U >= 2, whose merged-row matvec keeps the
// next row's records in registers.
constexpr int kPersMinBlocks = 2;
__host__ __device__ constexpr int pers_threads(int U, bool st) { return (!st && U >= 2) ? 512 : 768; }
constexpr unsigned long long kSpinTimeoutNs = 2000000000ull;  // 2 s

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int *p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void red_release_add_u32(unsigned int *p, unsigned int v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Bulk asynchronous copy global -> shared memory completing on an mbarrier
// (the copy engine, no registers); 16-byte aligned addresses and sizes.
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0u;
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Sum of NV accumulators over the CTA in a fixed tree order; the result is
// valid in thread 0.  sh: one slot per warp.
template <typename R, int NV>
__device__ __forceinline__ void cta_sum(typename Acc<R>::T (&v)[NV], typename Acc<R>::T (*sh)[NV]) {
  typedef Acc<R> A;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] = A::add(v[k], A::shfl(v[k], o));
    if (lane == 0) sh[wid][k] = v[k];
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      v[k] = lane < nw ? sh[lane][k] : A::zero();
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v[k] = A::add(v[k], A::shfl(v[k], o));
    }
  }
  __syncthreads();  // sh is free again
}

// The CTA sums the gridDim.x partials of the barrier just passed in a fixed
// order: thread t of the first kPartWarps warps takes partials t, t + 256,
// ... (all its loads in flight: one L2 round trip for up to 512 CTAs), each
// warp folds its lanes by a shuffle tree, and thread 0 adds the warps' sums
// in warp order into tot.  Every CTA runs the same order, so all hold
// bit-identical totals.  Called by every thread of the CTA (blockDim.x >=
// 32 kPartWarps); sh is a free [>= kPartWarps][NV] scratch, free again on
// return.
constexpr int kPartWarps = 8;
__device__ __forceinline__ void put_tot(double &d, double v) { d = v; }
__device__ __forceinline__ void put_tot(double &d, DF v) { d = Acc<float>::to_d(v); }
__device__ __forceinline__ void put_tot(DF &d, DF v) { d = v; }

// tot: double, or DF to keep FP32-mode totals double-word (no FP64).
template <typename R, int NV, typename TOT>
__device__ __forceinline__ void grid_partials(const double *part, TOT *tot, typename Acc<R>::T (*sh)[NV],
                                              int nbg = -1) {
  typedef Acc<R> A;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nb = nbg < 0 ? (int)gridDim.x : nbg;
  constexpr int T = 32 * kPartWarps;
  if (wid < kPartWarps) {
    typename A::T w[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) w[k] = A::zero();
    for (int j0 = (int)threadIdx.x; j0 < nb; j0 += 2 * T) {
      typename A::T b0[NV], b1[NV];
      const int j1 = j0 + T;
#pragma unroll
      for (int k = 0; k < NV; ++k) {
        b0[k] = A::load(&part[(size_t)j0 * NV + k]);
        b1[k] = j1 < nb ? A::load(&part[(size_t)j1 * NV + k]) : A::zero();
      }
#pragma unroll
      for (int k = 0; k < NV; ++k) w[k] = A::add(A::add(w[k], b0[k]), b1[k]);
    }
#pragma unroll
    for (int k = 0; k < NV; ++k) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) w[k] = A::add(w[k], A::shfl(w[k], o));
      if (lane == 0) sh[wid][k] = w[k];
    }
  }
  __syncthreads();
  if (wid == 0) {  // the warps' sums folded by a shuffle tree in warp 0
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      typename A::T s = lane < kPartWarps ? sh[lane][k] : A::zero();
#pragma unroll
      for (int o = kPartWarps / 2; o > 0; o >>= 1) s = A::add(s, A::shfl(s, o));
      if (lane == 0) put_tot(tot[k], s);
    }
  }
  __syncthreads();  // sh is free again, tot is visible to every thread
}

struct NoHook {
  __device__ void operator()() const {}
};

// Grid all-reduce (see above).  part: this barrier's buffer of
// gridDim.x * NV slots; target: arrivals that complete this barrier.
// Returns false (in every thread) if the wait gave up; otherwise thread 0
// holds the totals in tot.  hook() runs in thread 0 as soon as the barrier
// has completed, before the partials are summed.  A group of CTAs (the
// CTAs of one plate of a batch) reduces among itself with cta = the CTA's
// rank in the group and nb = the group's size (defaults: the whole grid).
template <typename R, int NV, typename TOT, typename Hook = NoHook>
__device__ __forceinline__ bool grid_sum(typename Acc<R>::T (&v)[NV], double *part, SolveScalars *S,
                                         unsigned int target, TOT *tot, typename Acc<R>::T (*sh)[NV],
                                         int *ok_sh, const Hook &hook = Hook(), int cta = -1, int nb = -1) {
  typedef Acc<R> A;
  cta_sum<R, NV>(v, sh);  // its barriers order every thread's row writes before thread 0's release
  if (threadIdx.x == 0) {
    const int slot = cta < 0 ? (int)blockIdx.x : cta;
#pragma unroll
    for (int k = 0; k < NV; ++k) A::store(&part[(size_t)slot * NV + k], v[k]);
    red_release_add_u32(&S->bar, 1u);
    int ok = 1;
    const unsigned long long t0 = global_ns();
    unsigned int spins = 0;
    while (ld_acquire_u32(&S->bar) < target) {
      if ((++spins & 31u) == 0u) {  // another CTA gave up, or this wait is too long
        if (*(volatile int32_t *)&S->abort) {
          ok = 0;
          break;
        }
        if (global_ns() - t0 > kSpinTimeoutNs) {
          *(volatile int32_t *)&S->abort = 1;
          ok = 0;
          break;
        }
      }
    }
    if (ok) hook();
    *ok_sh = ok;
  }
  __syncthreads();
  if (!*ok_sh) return false;
  grid_partials<R, NV>(part, tot, sh, nb);
  return true;
}

// The solve's scalars, kept in shared memory by thread 0 of every CTA
// (identical in all CTAs); coef holds alpha and beta in the kernel
// precision for every thread.
// The two-all-reduce loops' scalar type: FP64 for FP64 meshes, double-word
// FP32 for FP32 meshes (no FP64 instruction in the loop; see fused_scalars).
template <typename R> struct Sc;
template <> struct Sc<double> {
  typedef double T;
  static __device__ __forceinline__ T from(double d) { return d; }
  static __device__ __forceinline__ double to(T v) { return v; }
  static __device__ __forceinline__ T div(T a, T b) { return a / b; }
  static __device__ __forceinline__ bool zero(T a) { return a == 0.0; }
  static __device__ __forceinline__ bool finite(T a) { return !isnan(a) && !isinf(a); }
  static __device__ __forceinline__ double coef(T a) { return a; }
  // ||r|| <= tol ||b_eff||, as the kernel-per-phase loop takes it
  static __device__ __forceinline__ bool stop(T t0, double tol, double bn, T) { return sqrt(t0) <= tol * bn; }
};
template <> struct Sc<float> {
  typedef DF T;
  static __device__ __forceinline__ T from(double d) { return df_from(d); }
  static __device__ __forceinline__ double to(T v) { return df_to(v); }
  static __device__ __forceinline__ T div(T a, T b) { return df_div(a, b); }
  static __device__ __forceinline__ bool zero(T a) { return a.hi == 0.f; }
  static __device__ __forceinline__ bool finite(T a) { return df_finite(a); }
  static __device__ __forceinline__ float coef(T a) { return a.hi; }
  // |r|^2 <= (tol ||b_eff||)^2 (thr2)
  static __device__ __forceinline__ bool stop(T t0, double, double, T thr2) { return df_le(t0, thr2); }
};

template <typename R> struct PersShared {
  typedef typename Sc<R>::T T;
  T rho, beta, alpha, rr, pq, thr2;
  double bn;
  T tot[2];
  int iters, status, done, flag, ok;
  R coef[2];
};

// Thread 0: the two-all-reduce loops' scalars at the start, alpha after the
// p.q all-reduce (false: p = 0, the iterate is exact), the stop test and
// beta after the (|r|^2, r.z) all-reduce (true: stop), and the scalars left
// for the kernel-per-phase loop at the end.
template <typename R>
__device__ __forceinline__ void pers_load(PersShared<R> &z, const SolveScalars *S, double tol) {
  typedef Sc<R> C;
  z.rho = C::from(S->rho);
  z.beta = C::from(S->beta);
  z.alpha = C::from(S->alpha);
  z.rr = C::from(S->rr);
  z.pq = C::from(S->pq);
  z.bn = S->bn;
  z.thr2 = C::from(tol * S->bn * (tol * S->bn));
  z.iters = S->iters;
  z.status = kStOk;
  z.done = 0;
  z.coef[1] = sizeof(R) == 4 ? (R)S->beta_f : (R)S->beta;
}

template <typename R>
__device__ __forceinline__ bool pers_alpha(PersShared<R> &z) {
  typedef Sc<R> C;
  z.pq = z.tot[0];
  if (C::zero(z.pq)) return false;
  z.alpha = C::div(z.rho, z.pq);
  z.coef[0] = (R)C::coef(z.alpha);
  return true;
}

template <typename R>
__device__ __forceinline__ bool pers_beta(PersShared<R> &z, double tol, int max_it) {
  typedef Sc<R> C;
  bool stop = false;
  const typename C::T t0 = z.tot[0], t1 = z.tot[1];
  z.iters += 1;
  z.rr = t0;
  if (!C::finite(t0)) {
    z.status = kStNonfinite;
    z.done = 1;
    stop = true;
  } else if (C::stop(t0, tol, z.bn, z.thr2)) {
    z.done = 1;
    stop = true;
  }
  if (!stop && z.iters >= max_it) {
    stop = true;
    z.status = kStNotConverged;
    z.done = 1;
  }
  z.beta = !C::zero(z.rho) ? C::div(t1, z.rho) : C::from(0.0);
  z.rho = t1;
  z.coef[1] = (R)C::coef(z.beta);
  return stop;
}

template <typename R>
__device__ __forceinline__ void pers_store(PersShared<R> &z, SolveScalars *S) {
  typedef Sc<R> C;
  if (!z.ok) {
    z.status = kStTimeout;
    z.done = 1;
  }
  S->iters = z.iters;
  S->rr = C::to(z.rr);
  S->pq = C::to(z.pq);
  S->alpha = C::to(z.alpha);
  S->alpha_f = (float)C::coef(z.alpha);
  S->beta = C::to(z.beta);
  S->beta_f = (float)C::coef(z.beta);
  S->rho = C::to(z.rho);
  S->status = z.status;
  S->done = z.done;
}

// Partials: P.part holds two buffers of 2 * gridDim.x slots, used by
// alternate barriers (a CTA can only refill a buffer after every CTA has
// passed the barrier that read it).  ST (FP32): the CTA first copies the
// element records and history of its rows' elements into shared memory
// (bulk asynchronous copies, one mbarrier, bounded wait) and every matvec
// reads them there: the operator data cross the memory system once per
// solve instead of once per iteration.
template <typename R, int U, bool ST>
__global__ void __launch_bounds__(pers_threads(U, ST), kPersMinBlocks) k_cg_persistent(Params<R> P) {
  typedef Acc<R> AC;
  SolveScalars *S = P.sc;
  __shared__ typename AC::T sh[pers_threads(U, ST) / 32][2];
  __shared__ PersShared<R> z;
  __shared__ __align__(8) unsigned long long stage_bar;
  extern __shared__ __align__(128) unsigned char stage_smem[];
  if (S->done) return;  // set-up found b_eff = 0 or r_0 already small
  int row0 = 0, row1 = 0;
  const float4 *srec = nullptr;
  const float *sH = nullptr;
  if constexpr (ST) {
    const StageCta sc = P.st_cta[blockIdx.x];
    const int nel = sc.nel;
    row0 = sc.row0;
    row1 = sc.row1;
    srec = reinterpret_cast<const float4 *>(stage_smem);
    sH = reinterpret_cast<const float *>(stage_smem + (size_t)nel * sizeof(ERec<float>));
    if (threadIdx.x == 0) {
      mbar_init(&stage_bar, 1);
      const int r0 = sc.r0, r1 = sc.r1;
      mbar_arrive_expect_tx(&stage_bar, (unsigned)nel * (unsigned)(sizeof(ERec<float>) + sizeof(float)));
      unsigned off = 0;
      for (int r = r0; r < r1; ++r) {
        const int2 g = P.st_rng[r];  // first element (a multiple of 4), count (a multiple of 4)
        bulk_g2s(stage_smem + (size_t)off * sizeof(ERec<float>), P.rec + g.x, (unsigned)g.y * sizeof(ERec<float>),
                 &stage_bar);
        bulk_g2s((void *)(sH + off), P.Hr + g.x, (unsigned)g.y * sizeof(float), &stage_bar);
        off += (unsigned)g.y;
      }
    }
    __syncthreads();  // the barrier is initialised before anyone polls it
    bool ok = true;
    const unsigned long long t0 = global_ns();
    unsigned spins = 0;
    while (!mbar_try_wait(&stage_bar, 0u)) {
      if ((++spins & 15u) == 0u && global_ns() - t0 > kSpinTimeoutNs) {
        ok = false;
        break;
      }
    }
    if (!ok) *(volatile int32_t *)&S->abort = 1;
    if (threadIdx.x == 0) z.ok = 1;
    __syncthreads();
    if (!ok) z.ok = 0;
    __syncthreads();
    if (!z.ok) {
      if (blockIdx.x == 0 && threadIdx.x == 0) {
        S->status = kStTimeout;
        S->done = 1;
        S->inner_done = 1;
      }
      return;
    }
  }
  if (threadIdx.x == 0) pers_load(z, S, P.tol);
  __syncthreads();
  const unsigned int nb = gridDim.x;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
  unsigned int nbar = 0;
  for (;;) {
    // q = A p_new, p_new . q
    typename AC::T v1[1] = {AC::zero()};
    if constexpr (ST)
      matvec_rows_staged<U>(P, z.coef[1], row0, row1, srec, sH, v1[0]);
    else
      matvec_rows<R, U>(P, z.coef[1], tid, stride, v1[0], -1, (z.iters & 1) != 0);
    ++nbar;
    if (!grid_sum<R, 1>(v1, P.part + (nbar & 1u) * 2u * nb, S, nbar * nb + P.bar_extra, z.tot,
                        (typename AC::T(*)[1])sh, &z.ok))
      break;
    if (threadIdx.x == 0) {
      const bool moved = pers_alpha(z);  // p = 0: nothing moved, the iterate is exact
      z.done = moved ? z.done : 1;
      z.flag = moved ? 0 : 1;
    }
    __syncthreads();
    if (z.flag) break;
    // x += alpha p, r -= alpha q, z = r / diag; |r|^2 and r.z
    typename AC::T v3[3] = {AC::zero(), AC::zero(), AC::zero()};
    bool proj = false;
    update_rows<R>(P, z.coef[0], z.coef[1], tid, stride, v3, proj, -1, (z.iters & 1) != 0);
    typename AC::T v2[2] = {v3[0], v3[1]};
    ++nbar;
    if (!grid_sum<R, 2>(v2, P.part + (nbar & 1u) * 2u * nb, S, nbar * nb + P.bar_extra, z.tot, sh, &z.ok))
      break;
    if (threadIdx.x == 0) z.flag = pers_beta(z, P.tol, P.max_it) ? 1 : 0;
    __syncthreads();
    if (z.flag) break;
  }
  // CTA 0 leaves the scalars as the kernel-per-phase loop would
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    pers_store(z, S);
    S->inner_done = 1;
  }
}

// ------------------------------------ single-reduction persistent CG
//
// Jacobi PCG in the recurrences of Chronopoulos and Gear (1989): with
// u = M^-1 r, w = A u and s = A p carried as vectors, both inner products
// of an iteration, gamma = (r, u) and delta = (w, u), come from the same
// pass, so each iteration is one pass over the rows and one grid
// all-reduce instead of two of each:
//   p = u + beta p,  s = w + beta s,  x += alpha p,  r -= alpha s,
//   u = M^-1 r,  w = A u,  gamma' = (r, u),  delta' = (w, u),
//   beta' = gamma' / gamma,  alpha' = gamma' / (delta' - beta' gamma' / alpha).
// A row's matvec needs its neighbours' new u before they are stored: every
// row rebuilds it from the neighbour's (r, w, s, 1/diag) of the previous
// pass, which is why those four live in one 16-byte record, double
// buffered.  In exact arithmetic the iterates are those of the Jacobi PCG
// of the kernel-per-phase loop; the stop test is the same (||r|| <= tol
// ||b_eff||, r carried by the recurrence).  Set-up: copy (r0, 0, 0, 1/diag)
// from the right-hand side kernel's output, then one pass with
// alpha = beta = 0 gives w0 = A u0 and delta0.  FP32 only.

__device__ __forceinline__ float cg_unew(const float4 v, float al, float be) {
  return v.w * fmaf(-al, fmaf(be, v.z, v.y), v.x);
}

// Width-6 merged rows of one single-reduction pass, software-pipelined as
// nb_rows6 (the next row's records load while this row's neighbours are
// gathered); the arithmetic of fused_rows.
__device__ __forceinline__ void fused_rows6(const Params<float> &P, float al, float be,
                                            const float4 *__restrict__ vin, float4 *__restrict__ vout, int i0,
                                            int stride, DF (&acc)[3], bool rev) {
  typedef Acc<float> AC;
  const int jlast = i0 < P.N ? i0 + (P.N - 1 - i0) / stride * stride : i0 - stride;
  const int step = rev ? -stride : stride;
  NbRow6 cur;
  if (i0 < P.N) nb_load6(P, rev ? jlast : i0, cur);
  for (int j = rev ? jlast : i0; rev ? j >= i0 : j < P.N; j += step) {
    NbRow6 nxt;
    const int jn = j + step;
    if (rev ? jn >= i0 : jn < P.N) nb_load6(P, jn, nxt);
    const float4 v = vin[j];
    if ((cur.fl & kNotch) || (P.freef && !P.freef[j])) {  // eliminated row: everything stays zero
      vout[j] = make_float4(0.f, 0.f, 0.f, 0.f);
      cur = nxt;
      continue;
    }
    const float p = fmaf(be, P.cgp[j], v.w * v.x);
    const float sn = fmaf(be, v.z, v.y);
    const float rn = fmaf(-al, sn, v.x);
    const float un = v.w * rn;
    P.x[j] = fmaf(al, p, P.x[j]);
    P.cgp[j] = p;
    float wq = cur.dg * un;
    float u[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const uint32_t x = cur.w[k >> 1];
      const int o = (k & 1) ? (int)x >> 16 : (int)(int16_t)(x & 0xffffu);
      u[k] = cg_unew(vin[j + o], al, be);
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) wq = fmaf(cur.c[k], u[k], wq);
    vout[j] = make_float4(rn, wq, sn, v.w);
    const float sr = P.rscale * rn;
    acc[0] = AC::add(acc[0], AC::prod(sr, un));             // gamma
    acc[1] = AC::add(acc[1], AC::prod(P.rscale * wq, un));  // delta
    acc[2] = AC::add(acc[2], AC::prod(sr, sr));             // |r|^2
    cur = nxt;
  }
}

// Rows i0, i0 + stride, ... < N of one single-reduction pass, operator and
// neighbour vectors read from global memory (U entries in flight; merged
// rows of width 6: U >= 2 pipelines rows).
// Element-wise rows of one single-reduction pass with shared gathers
// (el_rows6's operator, fused_rows6's recurrences).
__device__ __forceinline__ void fused_el_rows6(const Params<float> &P, float al, float be,
                                               const float4 *__restrict__ vin, float4 *__restrict__ vout, int i0,
                                               int stride, DF (&acc)[3], bool rev) {
  typedef Acc<float> AC;
  const int jlast = i0 < P.N ? i0 + (P.N - 1 - i0) / stride * stride : i0 - stride;
  const int step = rev ? -stride : stride;
  for (int j = rev ? jlast : i0; rev ? j >= i0 : j < P.N; j += step) {
    ElRow6 cur;
    el_load6(P, j, cur);
    const float4 v = vin[j];
    if ((cur.fl & kNotch) || (P.freef && !P.freef[j])) {  // eliminated row: everything stays zero
      vout[j] = make_float4(0.f, 0.f, 0.f, 0.f);
      continue;
    }
    const float p = fmaf(be, P.cgp[j], v.w * v.x);
    const float sn = fmaf(be, v.z, v.y);
    const float rn = fmaf(-al, sn, v.x);
    const float un = v.w * rn;
    P.x[j] = fmaf(al, p, P.x[j]);
    P.cgp[j] = p;
    float u[6];
    el_gather6(cur, j, u, [&](int n) { return cg_unew(vin[n], al, be); });
    const float wq = el_apply6(cur, u, un, cur.dg * un);
    vout[j] = make_float4(rn, wq, sn, v.w);
    const float sr = P.rscale * rn;
    acc[0] = AC::add(acc[0], AC::prod(sr, un));             // gamma
    acc[1] = AC::add(acc[1], AC::prod(P.rscale * wq, un));  // delta
    acc[2] = AC::add(acc[2], AC::prod(sr, sr));             // |r|^2
  }
}

template <int U>
__device__ __forceinline__ void fused_rows(const Params<float> &P, float al, float be, const float4 *__restrict__ vin,
                                           float4 *__restrict__ vout, int i0, int stride, DF (&acc)[3],
                                           bool rev = false) {
  typedef Acc<float> AC;
  if (U >= 2 && P.nbc && P.Dn <= 6) {
    fused_rows6(P, al, be, vin, vout, i0, stride, acc, rev);
    return;
  }
  if (U >= 2 && P.gnbo) {
    fused_el_rows6(P, al, be, vin, vout, i0, stride, acc, rev);
    return;
  }
  const int jlast = i0 < P.N ? i0 + (P.N - 1 - i0) / stride * stride : i0 - stride;
  const int jstep = rev ? -stride : stride;
  for (int j = rev ? jlast : i0; rev ? j >= i0 : j < P.N; j += jstep) {
    const float4 v = vin[j];
    if (is_fixed(P, j)) {  // eliminated row: everything stays zero
      vout[j] = make_float4(0.f, 0.f, 0.f, 0.f);
      continue;
    }
    const float p = fmaf(be, P.cgp[j], v.w * v.x);
    const float sn = fmaf(be, v.z, v.y);
    const float rn = fmaf(-al, sn, v.x);
    const float un = v.w * rn;
    P.x[j] = fmaf(al, p, P.x[j]);
    P.cgp[j] = p;
    // entry records (FP32 meshes always carry them; only the staged
    // families, which use local_rows, run without): diag_j u_j, then per
    // slot c_b u_b + c_c u_c with the neighbours' u rebuilt from their
    // records
    float wq = P.diag[j] * un;
    if (P.nbc) {
      wq = nb_row_any(P, j, wq, [&](int n) { return cg_unew(vin[n], al, be); });
    } else if (P.fno) {
      wq = fan_row(P, P.ecf, j, wq, [&](int n) { return cg_unew(vin[n], al, be); });
    } else if (P.ecmp) {
      for (int k = 0; k < P.D; k += U) {
        uint32_t w[U];
        float2 cf[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const bool in = k + u < P.D;
          w[u] = in ? __ldg(&P.ecmp[(size_t)(k + u) * P.N + j]) : 0u;
          cf[u] = in ? __ldg(&P.ecf[(size_t)(k + u) * P.N + j]) : make_float2(0.f, 0.f);
        }
        float c[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int ob = (int)(int16_t)(w[u] & 0xffffu), oc = (int)w[u] >> 16;
          c[u] = fmaf(cf[u].x, cg_unew(vin[j + ob], al, be), __fmul_rn(cf[u].y, cg_unew(vin[j + oc], al, be)));
        }
#pragma unroll
        for (int u = 0; u < U; ++u) wq = __fadd_rn(wq, c[u]);
      }
    } else {
      for (int k = 0; k < P.D; k += U) {
        float4 er[U];
#pragma unroll
        for (int u = 0; u < U; ++u)
          er[u] = k + u < P.D ? __ldg(&P.erec[(size_t)(k + u) * P.N + j]) : make_float4(__int_as_float(-1), 0.f, 0.f, 0.f);
        float c[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int nb = __float_as_int(er[u].x);
          if (nb >= 0)
            c[u] = fmaf(er[u].z, cg_unew(vin[nb], al, be), __fmul_rn(er[u].w, cg_unew(vin[__float_as_int(er[u].y)], al, be)));
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (__float_as_int(er[u].x) >= 0) wq = __fadd_rn(wq, c[u]);
      }
    }
    vout[j] = make_float4(rn, wq, sn, v.w);
    const float sr = P.rscale * rn;
    acc[0] = AC::add(acc[0], AC::prod(sr, un));             // gamma
    acc[1] = AC::add(acc[1], AC::prod(P.rscale * wq, un));  // delta
    acc[2] = AC::add(acc[2], AC::prod(sr, sr));             // |r|^2
  }
}

// The CTA's rows of one single-reduction pass with everything in shared
// memory: localized element records (n0 | n1 << 16, n2 as positions in vs,
// kappa A, (cbase + 2 H) A / 12, gradients), the rows' entries
// (slot[k * mc + row - row0]) and the neighbourhood's (r, w, s, 1/diag) in
// vs, own rows from position own.  The recurrences of fused_rows, with the
// operator rebuilt per entry from the localized records.
template <int U>
__device__ __forceinline__ void local_rows(const Params<float> &P, float al, float be, const float4 *vs, int own,
                                           int row0, int row1, const uint16_t *slot, int mc, const float4 *srec,
                                           float4 *__restrict__ vout, DF (&acc)[3]) {
  typedef Acc<float> AC;
  for (int jl = threadIdx.x; jl < row1 - row0; jl += blockDim.x) {
    const int j = row0 + jl;
    const float4 v = vs[own + jl];
    if (is_fixed(P, j)) {
      vout[j] = make_float4(0.f, 0.f, 0.f, 0.f);
      continue;
    }
    const float p = fmaf(be, P.cgp[j], v.w * v.x);
    const float sn = fmaf(be, v.z, v.y);
    const float rn = fmaf(-al, sn, v.x);
    const float un = v.w * rn;
    P.x[j] = fmaf(al, p, P.x[j]);
    P.cgp[j] = p;
    float wq = 0.f;
    for (int k = 0; k < P.D; k += U) {
      float c[U];
      unsigned sl[U];
#pragma unroll
      for (int u = 0; u < U; ++u) sl[u] = k + u < P.D ? (unsigned)slot[(k + u) * mc + jl] : 0xffffu;
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (sl[u] == 0xffffu) continue;
        const int sidx = (int)(sl[u] >> 2), a = (int)(sl[u] & 3u);
        const float4 r0 = srec[2 * sidx], G = srec[2 * sidx + 1];
        const unsigned n01 = __float_as_uint(r0.x);
        const float u0 = a == 0 ? un : cg_unew(vs[n01 & 0xffffu], al, be);
        const float u1 = a == 1 ? un : cg_unew(vs[n01 >> 16], al, be);
        const float u2 = a == 2 ? un : cg_unew(vs[__float_as_int(r0.y)], al, be);
        c[u] = elem_row<float>(G, a, r0.z, r0.w, u0, u1, u2);
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (sl[u] != 0xffffu) wq = radd(wq, c[u]);
    }
    vout[j] = make_float4(rn, wq, sn, v.w);
    const float sr = P.rscale * rn;
    acc[0] = AC::add(acc[0], AC::prod(sr, un));
    acc[1] = AC::add(acc[1], AC::prod(P.rscale * wq, un));
    acc[2] = AC::add(acc[2], AC::prod(sr, sr));
  }
}

// CTA shape: global operator, two CTAs of 512 per SM; shared-memory operator,
// one CTA of 1024 per SM (the staged share of an SM is one CTA's); 32 warps
// per SM and at most 64 registers either way.
template <bool ST> struct FusedCfg {
  static constexpr int threads = ST ? 1024 : 512;
  static constexpr int minb = ST ? 1 : 2;
};

// CTA size and residency of the unstaged single-reduction kernel per
// variant U: 512 threads (64 registers) for U <= 2, 384 for U = 3 and 256
// (three per SM) for U = 4 -- up to 85 registers, for rows whose records
// and neighbour values do not fit 64 (the element-wise rows).  The
// autotuner times every variant.
__host__ __device__ constexpr int fused_threads(int U, bool ST) {
  return ST ? FusedCfg<true>::threads : (U == 3 ? 384 : U == 4 ? 256 : FusedCfg<false>::threads);
}
__host__ __device__ constexpr int fused_minb(int U, bool ST) {
  return ST ? FusedCfg<true>::minb : (U == 4 ? 3 : 2);
}

struct FusedShared {
  DF gamma, alpha, rr, thr2;  // double-word: no FP64 instruction in the loop
  DF tot[3];
  int iters, status, done, flag, ok;
  float al, be;
};

// Thread 0 of every CTA: the solve's scalars at the start of the loop; the
// stop test ||r|| <= tol ||b_eff|| is taken as |r|^2 <= (tol ||b_eff||)^2.
__device__ __forceinline__ void fused_load(FusedShared &z, const SolveScalars *S, double tol) {
  const double t = tol * S->bn;
  z.thr2 = df_from(t * t);
  z.gamma = df_from(S->rho);
  z.rr = df_from(S->rr);
  z.iters = S->iters;
  z.status = kStOk;
  z.done = 0;
  z.al = 0.f;
  z.be = 0.f;
  z.alpha = DF{0.f, 0.f};
}

// Thread 0 of every CTA after the all-reduce of pass `pass` (gamma, delta,
// |r|^2 in z.tot): the stop tests and the next alpha and beta of the
// single-reduction recurrences, in double-word arithmetic; z.flag = 1 ends
// the loop.
__device__ __forceinline__ void fused_scalars(FusedShared &z, const Params<float> &P, int pass) {
  const DF g1 = z.tot[0], d1 = z.tot[1], t0 = z.tot[2];
  bool stop = false;
  if (pass > 1) {  // pass 1 was the set-up pass (w0 = A u0): no iterate yet
    z.iters += 1;
    z.rr = t0;
  }
  if (!df_finite(t0) || !df_finite(d1)) {
    z.status = kStNonfinite;
    z.done = 1;
    stop = true;
  } else if (pass > 1 && df_le(t0, z.thr2)) {
    z.done = 1;
    stop = true;
  } else if (g1.hi == 0.f) {  // u = 0: the iterate is exact
    z.done = 1;
    stop = true;
  }
  if (!stop && z.iters >= P.max_it) {
    stop = true;
    z.status = kStNotConverged;
    z.done = 1;
  }
  if (!stop) {
    const DF beta = pass > 1 ? df_div(g1, z.gamma) : DF{0.f, 0.f};
    const DF den = pass > 1 ? df_sub(d1, df_mul(beta, df_div(g1, z.alpha))) : d1;
    const DF alpha = df_div(g1, den);
    if (den.hi == 0.f || !df_finite(den) || !df_finite(alpha)) {  // breakdown: A is SPD, so only through rounding
      z.status = kStNonfinite;
      z.done = 1;
      stop = true;
    } else {
      z.alpha = alpha;
      z.gamma = g1;
      z.al = alpha.hi;
      z.be = beta.hi;
    }
  }
  z.flag = stop ? 1 : 0;
}

// CTA 0's thread 0 at the end: the scalars as the kernel-per-phase loop
// leaves them.
__device__ __forceinline__ void fused_store(FusedShared &z, SolveScalars *S) {
  if (!z.ok) {
    z.status = kStTimeout;
    z.done = 1;
  }
  S->iters = z.iters;
  S->rr = df_to(z.rr);
  S->rho = df_to(z.gamma);
  S->alpha = df_to(z.alpha);
  S->status = z.status;
  S->done = z.done;
  S->inner_done = 1;
}

// Shared-memory layout of the local (ST) kernel for one CTA: element
// records (32 B), row entries (D rows of mc = row count rounded up to 8),
// then a region that first receives the elements' history (4 B each) and,
// once the records have absorbed it, the neighbourhood's vectors (16 B
// each); byte offsets.
struct LocalLayout {
  unsigned slot, vec, total;
  int mc;
};

__host__ __device__ __forceinline__ LocalLayout local_layout(int nel, int rows, int D, int nn) {
  LocalLayout L;
  L.mc = (rows + 7) / 8 * 8;
  L.slot = (unsigned)nel * (unsigned)sizeof(ERec<float>);
  L.vec = (L.slot + (unsigned)D * (unsigned)L.mc * 2u + 15u) / 16u * 16u;
  const unsigned nv = (unsigned)nn * 16u, nh = (unsigned)nel * 4u;
  L.total = L.vec + (nv > nh ? nv : nh);
  return L;
}

__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long *bar, unsigned parity) {
  const unsigned long long t0 = global_ns();
  unsigned spins = 0;
  while (!mbar_try_wait(bar, parity))
    if ((++spins & 15u) == 0u && global_ns() - t0 > kSpinTimeoutNs) return false;
  return true;
}

// ST = false: rows read the operator and the neighbours' vectors from global
// memory.  ST = true (local): once per solve the CTA copies its localized
// element records, their history and its rows' entries into shared memory,
// and before every pass the (r, w, s, 1/diag) of every node its elements
// touch (bulk copies on two mbarriers, bounded waits); the pass itself then
// reads shared memory only and writes its rows' results to global memory.
template <int U, bool ST>
__global__ void __launch_bounds__(fused_threads(U, ST), fused_minb(U, ST)) k_cg_fused(Params<float> P) {
  typedef Acc<float> AC;
  SolveScalars *S = P.sc;
  __shared__ DF sh[32][3];
  __shared__ FusedShared z;
  __shared__ __align__(8) unsigned long long bar_static, bar_vec;
  extern __shared__ __align__(128) unsigned char stage_smem[];
  if (S->done) return;  // set-up found b_eff = 0 or r_0 already small
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
  StageCta sc{};
  LocalLayout L{};
  if constexpr (ST) {
    sc = P.st_cta[blockIdx.x];
    L = local_layout(sc.nel, sc.row1 - sc.row0, P.D, sc.nn);
    if (threadIdx.x == 0) {
      mbar_init(&bar_static, 1);
      mbar_init(&bar_vec, 1);
      mbar_arrive_expect_tx(&bar_static, L.slot + (unsigned)sc.nel * 4u + (unsigned)P.D * (unsigned)L.mc * 2u);
      bulk_g2s(stage_smem, P.st_lrec + sc.lrec, L.slot, &bar_static);
      unsigned off = 0;
      for (int r = sc.r0; r < sc.r1; ++r) {
        const int2 g = P.st_rng[r];  // first element and count, multiples of 4
        bulk_g2s(stage_smem + L.vec + off * 4u, P.Hr + g.x, (unsigned)g.y * 4u, &bar_static);
        off += (unsigned)g.y;
      }
      for (int k = 0; k < P.D; ++k)
        bulk_g2s(stage_smem + L.slot + (unsigned)k * (unsigned)L.mc * 2u,
                 P.st_slot + (size_t)k * P.st_ns + sc.row0, (unsigned)L.mc * 2u, &bar_static);
    }
  }
  // set-up: (r0, 0, 0, 1/diag) and p = 0
  for (int j = tid; j < P.N; j += stride) {
    P.cgv0[j] = make_float4(P.r[j], 0.f, 0.f, P.dinv[j]);
    P.cgp[j] = 0.f;
  }
  if (threadIdx.x == 0) fused_load(z, S, P.tol);
  if constexpr (ST) {
    __syncthreads();  // the mbarriers are initialised before anyone polls them
    if (!mbar_wait_bounded(&bar_static, 0u)) *(volatile int32_t *)&S->abort = 1;  // all leave at the next barrier
    // records absorb the history: (n0 | n1 << 16, n2, kappa A, (cbase + 2 H) A / 12, grad)
    float4 *srec = reinterpret_cast<float4 *>(stage_smem);
    const float *hs = reinterpret_cast<const float *>(stage_smem + L.vec);
    for (int e = threadIdx.x; e < sc.nel; e += blockDim.x) {
      const float4 r0 = srec[2 * e];
      const float A = r0.w, h = hs[e];
      const float kA = P.kappa * A;
      const float mA = (P.cbase + 2.f * h) * A * (1.f / 12.f);
      const unsigned n01 = ((unsigned)__float_as_int(r0.x) & 0xffffu) | ((unsigned)__float_as_int(r0.y) << 16);
      srec[2 * e] = make_float4(__uint_as_float(n01), r0.z, kA, mA);
    }
    // the history region becomes the vectors' (async copies) after the
    // grid barrier below, which all threads reach after their reads
  }
  const unsigned int nb = gridDim.x;
  unsigned int nbar = 1;
  // ST: the copy of the neighbourhood's vectors for a pass is issued as
  // soon as the barrier before it completes (the rows it reads are written),
  // ahead of the partial sums.  The rows written in the last pass by other
  // CTAs (generic proxy, ordered before this thread by the barrier) are read
  // by the copy engine, which also overwrites shared memory this CTA last
  // read generically: hence the proxy fences.
  float4 *vs = ST ? reinterpret_cast<float4 *>(stage_smem + L.vec) : nullptr;
  int copies = 0;  // vector copies issued (ST)
  auto issue_vec = [&](const float4 *src) {
    if constexpr (ST) {
      asm volatile("fence.proxy.async.global;" ::: "memory");
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive_expect_tx(&bar_vec, (unsigned)sc.nn * 16u);
      unsigned off = 0;
      for (int r = sc.n0; r < sc.n1; ++r) {
        const int2 g = P.st_nrng[r];  // first node, count
        bulk_g2s(vs + off, src + g.x, (unsigned)g.y * 16u, &bar_vec);
        off += (unsigned)g.y;
      }
    }
  };
  DF v3[3] = {AC::zero(), AC::zero(), AC::zero()};
  bool fine = grid_sum<float, 3>(v3, P.part + 3u * nb, S, nb + P.bar_extra, z.tot, sh, &z.ok,
                                 [&]() { issue_vec(P.cgv0); });
  if (ST && fine) copies = 1;
  int pass = 0;  // passes read cgv[pass & 1] and write the other buffer
  while (fine) {
    float4 *vin = (pass & 1) ? P.cgv1 : P.cgv0;
    float4 *vout = (pass & 1) ? P.cgv0 : P.cgv1;
    DF acc[3] = {AC::zero(), AC::zero(), AC::zero()};
    if constexpr (ST) {
      if (!mbar_wait_bounded(&bar_vec, (unsigned)pass & 1u)) *(volatile int32_t *)&S->abort = 1;
      local_rows<U>(P, z.al, z.be, vs, sc.own, sc.row0, sc.row1,
                    reinterpret_cast<const uint16_t *>(stage_smem + L.slot), L.mc,
                    reinterpret_cast<const float4 *>(stage_smem), vout, acc);
    } else {
      fused_rows<U>(P, z.al, z.be, vin, vout, tid, stride, acc, (pass & 1) != 0);  // alternate directions
    }
    ++nbar;
    ++pass;
    if (ST) __syncthreads();  // every thread is done with vs before the next copy lands there
    if (!grid_sum<float, 3>(acc, P.part + (nbar & 1u) * 3u * nb, S, nbar * nb + P.bar_extra, z.tot, sh, &z.ok,
                            [&]() { issue_vec(vout); }))
      break;
    if (ST) copies = pass + 1;
    if (threadIdx.x == 0) fused_scalars(z, P, pass);
    __syncthreads();
    if (z.flag) break;
  }
  if constexpr (ST) {
    // a vector copy issued for a pass that did not run: let it land before
    // the CTA (and its shared memory) goes away
    if (copies > pass && !mbar_wait_bounded(&bar_vec, (unsigned)pass & 1u)) *(volatile int32_t *)&S->abort = 1;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) fused_store(z, S);
}

// ------------------------------------------- resident single-reduction CG
//
// The recurrences of k_cg_fused on fan-order element-wise rows (FP32), with
// CTA b owning rows [b R, (b+1) R) for the whole solve (R = P.res_rows).
// Per row, x, p, the operator diagonal, the three fan words and the fan
// length (with the row's fixed flag) stay in the CTA's shared memory from
// the set-up to the end of the loop, so a pass reads from global memory
// only the row's entry coefficients and the (r, w, s, 1/diag) records of
// the row and its neighbours, and writes only the row's record; x is
// written back when the loop ends.  kResWords 4-byte words a row bound R,
// which decides on which meshes the family exists.  U picks the CTA shape:
// 1024 threads (one CTA per SM), 512 (two), 384 (two, up to 85 registers)
// or 256 (three).  Per row the arithmetic of fused_rows; the dot products'
// partial sums are grouped by CTA range instead of grid stride.
// FULL (meshes small enough, e.g. a quarter-million rows on 148 SMs): the
// rows' coefficient pairs and their (r, w, s, 1/diag) records (both
// buffers) live in shared memory as well, kResWordsFull words a row; a
// pass then reads global memory only for neighbours owned by another CTA,
// and writes a new record to global memory only for the rows within the
// mesh's element span (P.res_halo) of either end of its range.
// Shared-memory layout (words, R a multiple of 4): [0, 7R) the base words
// (x, p, diagonal, fan words 0..2, fan length | fixed << 8, each R long);
// FULL adds [7R, 19R) the coefficient pairs of fan positions 0..5 (R
// float2 each) and [19R, 27R) the two record buffers (R float4 each).
__host__ __device__ constexpr int res_threads(int U) {
  return U == 1 ? 1024 : (U == 2 ? 512 : (U == 3 ? 384 : 256));
}
__host__ __device__ constexpr int res_minb(int U) { return U == 1 ? 1 : (U == 4 ? 3 : 2); }
constexpr int kResWords = 7;  // x, p, diagonal, fan words 0..2, fan length | fixed << 8
constexpr int kResWordsFull = 27;  // + 6 coefficient pairs + 2 records

__device__ __forceinline__ void resident_rows(const Params<float> &P, float al, float be,
                                              const float4 *__restrict__ vin, float4 *__restrict__ vout, int row0,
                                              int nr, int R, uint32_t *rs, DF (&acc)[3], bool rev) {
  typedef Acc<float> AC;
  float *xs = reinterpret_cast<float *>(rs);
  float *ps = xs + R;
  const float *ds = ps + R;
  const uint32_t *fw = rs + 3 * R, *meta = rs + 6 * R;
  const int T = (int)blockDim.x, t = (int)threadIdx.x;
  const int llast = t < nr ? t + (nr - 1 - t) / T * T : t - T;
  const int lstep = rev ? -T : T;
  for (int l = rev ? llast : t; rev ? l >= t : l < nr; l += lstep) {
    const int j = row0 + l;
    const float4 v = vin[j];
    const uint32_t mt = meta[l];
    if (mt & 0x100u) {  // eliminated row: everything stays zero
      vout[j] = make_float4(0.f, 0.f, 0.f, 0.f);
      continue;
    }
    const float p = fmaf(be, ps[l], v.w * v.x);
    const float sn = fmaf(be, v.z, v.y);
    const float rn = fmaf(-al, sn, v.x);
    const float un = v.w * rn;
    xs[l] = fmaf(al, p, xs[l]);
    ps[l] = p;
    const uint32_t w[3] = {fw[l], fw[R + l], fw[2 * R + l]};
    const float wq = fan_row_w(P, P.ecf, j, ds[l] * un, w, (int)(mt & 0xffu),
                               [&](int n) { return cg_unew(vin[n], al, be); });
    vout[j] = make_float4(rn, wq, sn, v.w);
    const float sr = P.rscale * rn;
    acc[0] = AC::add(acc[0], AC::prod(sr, un));             // gamma
    acc[1] = AC::add(acc[1], AC::prod(P.rscale * wq, un));  // delta
    acc[2] = AC::add(acc[2], AC::prod(sr, sr));             // |r|^2
  }
}

// FULL: the rows of a pass with everything of the CTA's own rows in
// shared memory; rin / rout the shared record buffers (old, new).
__device__ __forceinline__ void resident_rows_full(const Params<float> &P, float al, float be,
                                                   const float4 *__restrict__ vin, float4 *__restrict__ vout,
                                                   int row0, int nr, int R, uint32_t *rs, const float4 *rin,
                                                   float4 *rout, DF (&acc)[3], bool rev) {
  typedef Acc<float> AC;
  float *xs = reinterpret_cast<float *>(rs);
  float *ps = xs + R;
  const float *ds = ps + R;
  const uint32_t *fw = rs + 3 * R, *meta = rs + 6 * R;
  const float2 *cfs = reinterpret_cast<const float2 *>(rs + 7 * R);
  const int T = (int)blockDim.x, t = (int)threadIdx.x;
  const int llast = t < nr ? t + (nr - 1 - t) / T * T : t - T;
  const int lstep = rev ? -T : T;
  for (int l = rev ? llast : t; rev ? l >= t : l < nr; l += lstep) {
    const int j = row0 + l;
    const float4 v = rin[l];
    const uint32_t mt = meta[l];
    // only rows within the span of either end of the range are read by
    // another CTA, from global memory
    const bool edge = l < P.res_halo || l >= nr - P.res_halo;
    if (mt & 0x100u) {  // eliminated row: everything stays zero
      rout[l] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (edge) vout[j] = make_float4(0.f, 0.f, 0.f, 0.f);
      continue;
    }
    const float p = fmaf(be, ps[l], v.w * v.x);
    const float sn = fmaf(be, v.z, v.y);
    const float rn = fmaf(-al, sn, v.x);
    const float un = v.w * rn;
    xs[l] = fmaf(al, p, xs[l]);
    ps[l] = p;
    const uint32_t w[3] = {fw[l], fw[R + l], fw[2 * R + l]};
    float2 cf[6];
    float nv[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      cf[k] = k < P.D ? cfs[k * R + l] : make_float2(0.f, 0.f);
      const int ln = l + fan_offset(w, k);
      nv[k] = cg_unew((unsigned)ln < (unsigned)nr ? rin[ln] : vin[row0 + ln], al, be);
    }
    const float wq = fan_sum(ds[l] * un, cf, nv, (int)(mt & 0xffu));
    const float4 rec = make_float4(rn, wq, sn, v.w);
    rout[l] = rec;
    if (edge) vout[j] = rec;
    const float sr = P.rscale * rn;
    acc[0] = AC::add(acc[0], AC::prod(sr, un));             // gamma
    acc[1] = AC::add(acc[1], AC::prod(P.rscale * wq, un));  // delta
    acc[2] = AC::add(acc[2], AC::prod(sr, sr));             // |r|^2
  }
}

template <int U, bool FULL>
__global__ void __launch_bounds__(res_threads(U), res_minb(U)) k_cg_resident(Params<float> P) {
  typedef Acc<float> AC;
  SolveScalars *S = P.sc;
  __shared__ DF sh[32][3];
  __shared__ FusedShared z;
  extern __shared__ __align__(16) uint32_t res_smem[];
  if (S->done) return;  // set-up found b_eff = 0 or r_0 already small
  const int R = P.res_rows;
  const int row0 = (int)blockIdx.x * R;
  const int nr = max(0, min(R, P.N - row0));
  float *xs = reinterpret_cast<float *>(res_smem);
  float4 *recs = reinterpret_cast<float4 *>(res_smem + 19 * R);  // FULL: two buffers of R
  // set-up: the rows' resident words, p = 0 and (r0, 0, 0, 1/diag)
  for (int l = threadIdx.x; l < nr; l += blockDim.x) {
    const int j = row0 + l;
    xs[l] = P.x[j];
    xs[R + l] = 0.f;
    xs[2 * R + l] = P.diag[j];
#pragma unroll
    for (int k = 0; k < 3; ++k) res_smem[(3 + k) * R + l] = __ldg(&P.fno[(size_t)k * P.N + j]);
    res_smem[6 * R + l] = (__ldg(&P.fmap[j]) >> 24) | (is_fixed(P, j) ? 0x100u : 0u);
    const float4 rec = make_float4(P.r[j], 0.f, 0.f, P.dinv[j]);
    P.cgv0[j] = rec;
    if constexpr (FULL) {
      float2 *cfs = reinterpret_cast<float2 *>(res_smem + 7 * R);
#pragma unroll
      for (int k = 0; k < 6; ++k) cfs[k * R + l] = k < P.D ? __ldg(&P.ecf[(size_t)k * P.N + j]) : make_float2(0.f, 0.f);
      recs[l] = rec;
    }
  }
  if (threadIdx.x == 0) fused_load(z, S, P.tol);
  const unsigned int nb = gridDim.x;
  unsigned int nbar = 1;
  DF v3[3] = {AC::zero(), AC::zero(), AC::zero()};
  bool fine = grid_sum<float, 3>(v3, P.part + 3u * nb, S, nb + P.bar_extra, z.tot, sh, &z.ok);
  int pass = 0;  // passes read cgv[pass & 1] and write the other buffer
  while (fine) {
    const float4 *vin = (pass & 1) ? P.cgv1 : P.cgv0;
    float4 *vout = (pass & 1) ? P.cgv0 : P.cgv1;
    DF acc[3] = {AC::zero(), AC::zero(), AC::zero()};
    if constexpr (FULL)
      resident_rows_full(P, z.al, z.be, vin, vout, row0, nr, R, res_smem, recs + (pass & 1) * R,
                         recs + ((pass + 1) & 1) * R, acc, (pass & 1) != 0);
    else
      resident_rows(P, z.al, z.be, vin, vout, row0, nr, R, res_smem, acc, (pass & 1) != 0);  // alternate directions
    ++nbar;
    ++pass;
    if (!grid_sum<float, 3>(acc, P.part + (nbar & 1u) * 3u * nb, S, nbar * nb + P.bar_extra, z.tot, sh, &z.ok))
      break;
    if (threadIdx.x == 0) fused_scalars(z, P, pass);
    __syncthreads();
    if (z.flag) break;
  }
  for (int l = threadIdx.x; l < nr; l += blockDim.x) P.x[row0 + l] = xs[l];
  if (blockIdx.x == 0 && threadIdx.x == 0) fused_store(z, S);
}

// AT1 restart (projected CG, Sec. 2.4): r = b - A x, active set
// {x <= lo, r <= 0} U {x >= hi, r >= 0}, free-set residual norm, a fresh
// direction p = z; converged when ||r_F|| <= tol ||b_eff||.
template <typename R>
__global__ void __launch_bounds__(256) k_at1_restart(Params<R> P) {
  typedef typename Params<R>::R4 R4;
  typedef Acc<R> AC;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R *cx = reinterpret_cast<R *>(smem_raw);
  typename AC::T vals[2] = {AC::zero(), AC::zero()};
  for (int b = blockIdx.x; b < P.nblk; b += gridDim.x) {
    int i0, i1, k0, k1;
    block_nodes(P, b, i0, i1, k0, k1);
    for (int k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
      const int en = __ldg(&P.ent[k]);
      const int e = en >> 2, a = en & 3;
      int4 t;
      R A;
      R4 G;
      load_elem(P, e, t, A, G);
      const R sg = gc_scale(P, e);
      const R kA = (P.kappa * sg) * A;
      const R mA = (P.cbase * sg + R(2) * P.Hr[e]) * A * (R(1) / R(12));
      cx[k - k0] = elem_row<R>(G, a, kA, mA, P.x[t.x], P.x[t.y], P.x[t.z]);
    }
    __syncthreads();
    for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
      if (P.flags[i] & kNotch) {
        P.freef[i] = 0;
        continue;
      }
      const int j0 = __ldg(&P.ptr[i]) - k0, j1 = __ldg(&P.ptr[i + 1]) - k0;
      R ax = 0;
      for (int j = j0; j < j1; ++j) ax += cx[j];
      const R xi = P.x[i], ri = P.b[i] - ax, lo = P.dprev[i];
      const bool act = (xi <= lo && ri <= R(0)) || (xi >= R(1) && ri >= R(0));
      P.r[i] = ri;
      P.freef[i] = act ? 0 : 1;
      typename Params<R>::R2 w;
      w.x = R(0);
      w.y = R(0);
      if (act) {
        P.pz[i] = w;
      } else {
        const R zi = ri * P.dinv[i];
        w.y = zi;
        P.pz[i] = w;
        const R sr = P.rscale * ri;
        vals[0] = AC::add(vals[0], AC::prod(sr, sr));
        vals[1] = AC::add(vals[1], AC::prod(sr, zi));
      }
    }
    __syncthreads();
  }
  __shared__ double tot[2];
  if (reduce_last<R, 2>(vals, P.part, P.ticket, tot) && threadIdx.x == 0) {
    SolveScalars &S = *P.sc;
    S.rr = tot[0];
    S.rho = tot[1];
    S.beta = 0.0;
    S.beta_f = 0.f;
    S.projected = 0;
    const bool conv = sqrt(tot[0]) <= P.tol * S.bn;
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
__global__ void __launch_bounds__(256) k_dmg_finish(Params<R> P) {
  // four nodes per thread and pass, every load before the first store
  // (d_out may alias d_prev: each node's store follows its own loads)
  constexpr int B = 4;
  const int stride = gridDim.x * blockDim.x;
  for (int i0 = blockIdx.x * blockDim.x + threadIdx.x; i0 < P.N; i0 += B * stride) {
    R x[B], lo[B];
    uint8_t fl[B];
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const int i = i0 + b * stride;
      if (i < P.N) {
        fl[b] = P.flags[i];
        x[b] = P.x[i];
        lo[b] = P.dprev[i];
      }
    }
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const int i = i0 + b * stride;
      if (i >= P.N) break;
      R v;
      if (fl[b] & kNotch) {
        v = R(1);
      } else {
        v = x[b];
        if (P.model == kAT2) {
          v = v > lo[b] ? v : lo[b];
          v = v < R(1) ? v : R(1);
        }
      }
      P.dout[i] = v;
    }
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

// End of a step without a damage solve (subcycling, Sec. 2.4): d stays d_n;
// the iteration log gets zeros and the step counter advances.
template <typename R>
__global__ void k_step_skip(Params<R> P) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (P.iters_log && P.step_ctr) {
      const int64_t n = *P.step_ctr;
      P.iters_log[2 * n] = 0;
      P.iters_log[2 * n + 1] = 0;
    }
    if (P.step_inc) *P.step_inc += 1;
  }
}

// ------------------------------------------------------------- energies

// E_el = sum A_e (g psi+ + psi-), E_frac per model (element loop), and
// E_kin = 1/2 sum m v^2 (node loop).  Terms in the kernel precision,
// accumulated in FP64 (double-word in FP32 mode).
template <typename R>
__global__ void __launch_bounds__(256) k_energies(Params<R> P) {
  typedef typename Params<R>::R2 R2;
  typedef typename Params<R>::R4 R4;
  typedef Acc<R> AC;
  typename AC::T vals[3] = {AC::zero(), AC::zero(), AC::zero()};
  const int stride = gridDim.x * blockDim.x;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < P.Ne; e += stride) {
    int4 t;
    R A;
    R4 G;
    load_elem(P, e, t, A, G);
    R exx, eyy, exy;
    elem_strain(P, G, t, exx, eyy, exy);
    const R d0 = P.d[t.x], d1 = P.d[t.y], d2 = P.d[t.z];
    const R db = (d0 + d1 + d2) * (R(1) / R(3));
    const R g = (R(1) - db) * (R(1) - db) + P.eta;
    R sxx, syy, sxy, psip;
    stress(P, exx, eyy, exy, R(1), sxx, syy, sxy, psip);
    // psi- = psi_full - psi+ for every split (psi_full = lambda/2 tr^2 + mu e:e)
    const R tr = exx + eyy;
    const R full = R(0.5) * P.lam * tr * tr + P.mu * (exx * exx + eyy * eyy + R(2) * exy * exy);
    const R psim = P.split == kIso ? R(0) : full - psip;
    vals[0] = AC::add(vals[0], AC::prod(A, g * psip + psim));
    const R gdx = G.x * (d0 - d2) + G.z * (d1 - d2);
    const R gdy = G.y * (d0 - d2) + G.w * (d1 - d2);
    const R g2 = gdx * gdx + gdy * gdy;
    const R Gc = (R)P.Gc * gc_scale(P, e), l0 = (R)P.l0;
    R dens;
    if (P.model == kAT1) {
      dens = Gc * R(0.375) * ((d0 + d1 + d2) * (R(1) / R(3)) / l0 + l0 * g2);
    } else {
      const R dMd = (R(2) * (d0 * d0 + d1 * d1 + d2 * d2) + R(2) * (d0 * d1 + d1 * d2 + d0 * d2)) * (R(1) / R(12));
      dens = Gc * (dMd / (R(2) * l0) + R(0.5) * l0 * g2);
    }
    vals[2] = AC::add(vals[2], AC::prod(A, dens));
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.N; i += stride) {
    const R2 vi = P.v[i];
    vals[1] = AC::add(vals[1], AC::prod(R(0.5) / P.minv[i], vi.x * vi.x + vi.y * vi.y));
  }
  __shared__ double tot[3];
  if (reduce_last<R, 3>(vals, P.part, P.ticket, tot) && threadIdx.x == 0) {
    P.energy_out[0] = tot[0];
    P.energy_out[1] = tot[1];
    P.energy_out[2] = tot[2];
    P.energy_out[3] = P.wext ? *P.wext : 0.0;
  }
}

}  // namespace pff
