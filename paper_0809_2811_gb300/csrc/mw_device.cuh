// mw_device.cuh -- device data layout and kernels of libmw (sm_103a).
//
// Model: Stillinger-Weber form with the mW parameters (Molinero & Moore,
// Sec. II.A and II.D):
//   E = sum_{i<j} phi2(r_ij) + sum_i sum_{j<k, legs of i} phi3(r_ij, r_ik, theta_jik)
//   phi2(r) = A eps [B (sig/r)^p - (sig/r)^q] exp(sig/(r - a sig))
//   phi3    = lam eps (cos th - cos th0)^2 exp(gam sig/(r - a sig)) exp(gam sig/(s - a sig))
// Dynamics: velocity Verlet with Berendsen or Nose-Hoover (Sec. II.B).
//
// Layout (all boxes concatenated box-major, atoms sorted by cell inside each
// box at every neighbour-list rebuild):
//   x,y,z            FP64 master positions as fractions of the box edge, [0, 1)
//   vx,vy,vz         FP64 master velocities (A/fs); between steps they lack the
//                    second half-kick of the last step (Global::pend), which
//                    the next kick1 folds into its own
//   q                uint4 {qx, qy, qz, box}: position as a 32-bit fraction of
//                    the box edge; the minimum-image difference of two atoms
//                    is the wrapping int32 difference, converted once to FP32
//   f                float4 forces (w unused), accumulated with red.global
//   nbr              int32 [N][W] neighbour list (atom-major rows), nbr_cnt[N]
//   cell_start       exclusive scan of atoms per cell, ncell + 1 entries
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace mw {

constexpr double kKB = 0.0019872042586408316;  // kcal/mol/K
constexpr double kFCONV = 4.184e-4;            // (kcal/mol/A)/(g/mol) -> A/fs^2
constexpr double kATM = 68568.4158;            // atm per kcal/mol/A^3
constexpr unsigned kFull = 0xffffffffu;

// Status codes written to Global::status (same values as mw_status).
enum : int { ST_OK = 0, ST_OVERFLOW = 3, ST_NAN = 4, ST_LOST = 5, ST_TIMEOUT = 6, ST_LEGS = 10, ST_GRID = 11,
             ST_CELLS = 12, ST_INPUT = 13 };

enum : int { TH_NVE = 0, TH_BERENDSEN = 1, TH_NH = 2, TH_NPT = 3 };

// Legs staged per centre atom in the fused force kernel's shared-memory table;
// centres with more legs take the overflow path.
constexpr int kLMax = 24;
// Upper bound for the overflow path (more legs than this = overlapping atoms).
constexpr int kMaxLegsOverflow = 64;

struct Box {        // read-only in kernels, except the geometry under isobaric runs (end_of_step_box)
  double L[3];
  double dtL[3];    // dt / L: drift of the box fraction per unit velocity
  float dtL64[3];   // dt / L * 2^64: drift in 2^-64 box-fraction units per unit velocity (FP32)
  float lost;       // half the shortest edge (A)
  double qs[3];     // 2^32 / L
  float Lq[3];      // L / 2^32
  int off, n;       // atom range
  int nc[3];        // cells per dimension
  int cell_off;     // first global cell
  double T0, Ndf, Q, volume;
  double invQ;      // 1 / Q
  double ndfkT0;    // N_df k_B T0
  double q4;        // dt / (4 Q): quarter-step factor of xi
  float q4f;        // q4 in FP32
  double inv_ndf_kb;  // 1 / (N_df k_B): T = 2 KE inv_ndf_kb
  double p_fac;     // atm per kcal/mol of 2 KE + tr W: 1/(3 V) in atm
  int vexp_lost;    // a velocity component whose FP32 exponent field is >= this is a runaway (see validate_integ)
  // isobaric runs only: the box scales at the drift of every step
  float hs2;        // squared displacement (measured with this step's Lq) that triggers a rebuild
  float a3;         // 1 + 3/N_df (barostat coupling)
  double W;         // barostat mass (N_df + 3) k_B T0 tau_p^2
  double Ln[3];     // edges of the coming step, made current by the last block of its kick1
};

struct BoxState {   // mutated by kernels
  float4 th;              // (xi hi, xi lo, eta hi, eta lo) after the start half of the next step
  float4 th_e;            // the same after the last end half
  double ke_last;         // KE after the last end half, or of the state just set (kcal/mol)
  double s_endc;          // last end scale, still pending on the stored velocities
  float sig;              // S - 1 for the next kick1: S = s_endc times the start-half scale
  int pad0_;
  double ke_acc[2];       // per step-parity raw kinetic energy of v + a (the second half-kick)
  double ew[2][8];        // per step-parity E2, E3, W[6]
  int rebuild;            // displacement flag of this box
  int pad_;
  long long rebuilds;
  double pe_b;            // barostat momentum (isobaric runs), after the start half of the next step
  double pe_e;            // the same after the last end half
  double Lb;              // edge 0 of the box at its last build (isotropic scaling: one ratio for all edges)
};

// Per-box thermo record written at the end of each step (doubles).
enum { TR_STEP, TR_PE, TR_E2, TR_E3, TR_KE, TR_T, TR_CONS, TR_P, TR_W0, TR_XI = TR_W0 + 6, TR_ETA,
       TR_REBUILDS, TR_VOL, TR_L0, TR_N = TR_L0 + 3 };

struct Global {
  unsigned long long step;  // completed steps since set_state
  int any_rebuild;
  int status;
  int max_count;            // widest neighbour set of the last build
  unsigned done;            // last-block counter of k_kick2
  int wpar;                 // parity slot of ew[] holding the virial of the latest force evaluation
  unsigned done1;           // last-block counter of k_kick1 (graph condition)
  long long rebuild_steps;  // steps (or force calls) that rebuilt at least one box
  int pend;                 // 1: velocities lack the second half-kick of the last step
  unsigned bar_count, bar_gen;  // persistent engine grid barrier
  int bar_stat[2];              // status snapshot taken at each barrier release
  long long npairs, ntrip;  // leg / triplet counts of the last force call (if counting)
  int count_terms;
  int n_over;               // centres routed to the overflow path
  int err_index;
  int pad_;
};

struct Integ {
  double dt;
  double cf;         // 0.5 dt FCONV / mass
  float cf_f;        // the same in FP32 (velocity increment = cf_f * F in FP32, added in FP64)
  double ke_fac;     // 0.5 mass / FCONV
  double tau;
  int kind;
  float half_skin2;  // (skin/2)^2
  double p_ext;      // target pressure of isobaric runs (kcal/mol/A^3)
  float skin, rlist; // list skin and radius (A): rebuild margin and cell check of a scaling box
};

// Cell grids of isobaric runs: laid out with cells kCellMargin r_list wide;
// a box that shrinks below r_list per cell, or grows so that one more cell
// of kCellGrow r_list fits, stops the run at a step boundary (ST_GRID) for
// the host to lay the grid out again.
constexpr double kCellMargin = 1.12;
constexpr double kCellGrow = 1.2;

// FP32 constants of the force kernels.  The *_lo fields hold the FP32
// rounding error of the constant before them (value = hi + lo to ~2^-48),
// which leg_terms adds back at first order.
struct FParams {
  float rc, rc2, rl2;
  float sig, sig_l2e, gsig_l2e, gsig;
  float Aeps, B, c0, sle;  // sle = sqrt(lambda eps)
  int p, q;
  float rc_lo, sig_lo, sig_l2e_lo, gsig_l2e_lo, B_lo;
};

// Several species: FP32 constants of the pair (a, b), from the parameter
// set of entry (a, b, b); the three-body leg factor of a leg from a centre
// of species a to one of species b uses the same set's gamma, sigma, a.
constexpr int kMaxSpecies = 8;
// h and c0 serve the moment kernel, for tables whose lambda epsilon of
// (centre a; legs b, c) is h_ab h_ac and whose cos theta0 depends on the
// centre alone: h = sqrt(lambda epsilon) of (a, b, b), c0 = cos theta0 of a.
struct SpPair {
  float rc, rc2, sig, sig_l2e, gsig, gsig_l2e, Aeps, B;
  int p, q;
  float h, c0;
  float rc_lo, sig_lo, sig_l2e_lo, gsig_l2e_lo, B_lo;  // as in FParams
};



struct Dev {
  int N, W, ncell, nbox;
  // master state: positions as 64-bit box fractions (s 2^64, wrapping), velocities
  // (A/fs) as unevaluated FP32 sums hi + lo (about 48 significant bits)
  unsigned long long *x, *y, *z;
  float2 *vx, *vy, *vz;
  unsigned long long *tx, *ty, *tz;
  float2 *tvx, *tvy, *tvz;
  int4 *img, *timg;   // periodic images crossed per component since the state was set (x, y, z)
  uint4 *q, *qb, *tq;
  float4* f;
  int *id, *tid;
  int *cell, *rank;
  int *cell_cnt, *cell_start;
  int* cell_box;      // box of each global cell
  int *nbr, *nbr_cnt;
  int* over;          // overflow centre list
  int* chunk;         // per-block cell totals of the persistent engine's scan
  int chunk_cap;
  const Box* box;
  BoxState* bst;
  double* thermo;     // nbox * TR_N
  Global* g;
  const Integ* integ;
  double* stage;      // n*3 doubles staging (user order)
  double* stage2;
  // several species (null / 1 for one species): species of each sorted atom
  // and its staging copy, the caller-order species, and the tables
  int *typ, *ttyp;
  const int* utyp;
  const SpPair* sp_pair;  // nsp^2, (a, b) at a nsp + b
  const float2* sp_tri;   // nsp^3: (lambda epsilon, cos theta0) of (centre a; legs b, c)
  int nsp;
  // phase marks of the persistent engine (null unless enabled): clock64 of
  // block 0 at kPhaseMarks points of each of the first marks_cap steps
  unsigned long long* marks;
  int marks_cap;
  // owner-computes force mode (null unless selected): per-atom moments of the
  // three-body terms (S0, s; M xx yy zz xy; M xz yz), the staged legs and
  // their count (-1: a centre over the staged-leg limit, done by scatter)
  float4* mom;
  int* legs;
  int* nleg;
};

constexpr int kPhaseMarks = 16;  // 14 used

// ---------------------------------------------------------------------------
// small helpers

__device__ __forceinline__ uint32_t to_fixed(double x, double qs) {
  return (uint32_t)(unsigned long long)__double2ll_rn(x * qs);
}

// 32-bit fixed-point coordinate of a 64-bit box fraction: round(s / 2^32)
// mod 2^32 (a fraction within half a unit of 1 wraps to 0).
__device__ __forceinline__ uint32_t q_of(unsigned long long s) {
  return (uint32_t)((s + 0x80000000ull) >> 32);
}

// Box fraction in [0, 1) (FP64) -> 64-bit fraction round(s 2^64) mod 2^64.
__device__ __forceinline__ unsigned long long frac64_of(double s) {
  const double t = s * 18446744073709551616.0;
  return (t >= 18446744073709551616.0) ? 0ull : __double2ull_rn(t);
}

// Exact conversion of an FP32 value to a 64-bit integer with integer
// operations only (no FP64 or 64-bit conversion instruction): |f| >= 2^23 is
// an integer already; smaller values round half away from zero; zero and
// subnormals give 0; magnitudes beyond 2^62 are clamped (a runaway atom,
// reported separately).
__device__ __forceinline__ long long f2ll_exact(float f) {
  const uint32_t u = __float_as_uint(f);
  const int ex = (int)((u >> 23) & 0xffu);
  const long long m = (long long)((u & 0x7fffffu) | 0x800000u);
  const int e = ex - 150;  // |f| = m 2^e
  long long r;
  if (ex == 0) r = 0;
  else if (e >= 0) r = m << min(e, 38);
  else if (e > -25) r = (m + (1ll << (-e - 1))) >> (-e);
  else r = 0;
  return (u >> 31) ? -r : r;
}

// Velocity as hi + lo (FP32 pair) <-> FP64 (set/get state and rare paths only).
__device__ __forceinline__ float2 split_df(double v) {
  const float hi = (float)v;
  return make_float2(hi, (float)(v - (double)hi));
}
__device__ __forceinline__ double join_df(float2 v) { return (double)v.x + (double)v.y; }

__device__ __forceinline__ float fix_diff(uint32_t a, uint32_t b, float lq) {  // b - a, minimum image
  return __int2float_rn((int)(b - a)) * lq;
}

// Store of v to *addr when p holds, as one predicated store (no branch
// around it).
__device__ __forceinline__ void st_if(bool p, int* addr, int v) {
  asm volatile("{\n .reg .pred q;\n setp.ne.b32 q, %0, 0;\n @q st.global.b32 [%1], %2;\n}" ::"r"((int)p), "l"(addr), "r"(v)
               : "memory");
}

__device__ __forceinline__ void red_add_v4(float4* addr, float a, float b, float c) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(a), "f"(b), "f"(c), "f"(0.0f)
               : "memory");
}

__device__ __forceinline__ float powi(float x, int n) {
  float r = 1.0f;
  for (int k = 0; k < n; ++k) r *= x;
  return r;
}

// ---------------------------------------------------------------------------
// One leg's terms (Sec. II.A) to about one FP32 ulp each.  The exponentials
// exp(sig/(r - a sig)) and exp(gam sig/(r - a sig)) amplify a relative error
// of their argument by the argument's size (about 2 at the first shell), and
// at the first shell the derivative of the pair term is a difference of two
// parts five to twenty times larger than itself (it vanishes at the phi2
// minimum).  So r, 1/r, 1/(r - a sig), the exponent arguments and the pair
// derivative carry their first-order corrections, which also absorb the
// error of the hardware approximations they start from:
//   r = r0 + dr, r0 = r2 rsqrt(r2), dr = (r2 - r0^2) / (2 r0) (residual by one FMA);
//   1/r = v (1 + ev), v = rsqrt(r2), ev = (1 - r0 v) - dr v;
//   x = r - a sig = (r0 - rc) + (dr - rc_lo) (r0 - rc exact for r0 >= rc / 2);
//   1/x = t (1 + tc), t ~ 1/(r0 - rc), tc = (1 - (r0 - rc) t) - (dr - rc_lo) t;
//   exp2(k / x) = exp2(k t) (1 + ln 2 (k t tc + RN residual of k t + k_lo t)).
// For the SW exponents (p, q) = (4, 0) the pair derivative
//   dphi2/dr = A eps e2 [(1 - y) sig / x^2 - 4 y / r],  y = B (sig / r)^4,
// is formed from hi + lo pairs (exact products by FMA, two-sum at the final
// difference); other exponents take the plain FP32 formula.  Returns false
// (nothing to add) when the leg is not inside a sig.
struct LegTerms {
  float r, invr;  // |d|, 1 / |d|
  float e3;       // exp(gam sig / (r - a sig))
  float nde;      // gam sig / (r - a sig)^2
  float phi;      // phi2(r)
  float dphi;     // dphi2 / dr
};

// 1/x from the hardware approximation (rcp.approx.ftz: within one ulp); the
// callers correct it to first order or need no more.
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
// 1/sqrt(x) and 2^x from the hardware approximations, subnormal inputs and
// results flushed to zero (the leg arithmetic corrects 1/sqrt to first order
// and the exponent's argument likewise; a 2^x below 2^-126 belongs to a leg at
// the cutoff, whose terms vanish there).
__device__ __forceinline__ float rsqrt_approx(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

template <class C>
__device__ __forceinline__ bool leg_terms(float r2, const C& c, LegTerms& o) {
  constexpr float kLn2 = 0.693147180559945f;
  const float v = rsqrt_approx(r2);
  const float r = r2 * v;
  const float dr = 0.5f * fmaf(-r, r, r2) * v;
  if (!(r + dr < c.rc)) return false;
  const float ev = fmaf(-r, v, 1.0f) - dr * v;
  const float xh = r - c.rc;
  const float xl = dr - c.rc_lo;
  const float t = rcp_approx(xh);  // < 0
  const float tc = fmaf(-xh, t, 1.0f) - xl * t;
  const float a2 = c.sig_l2e * t;
  const float a2l = fmaf(c.sig_l2e, t, -a2) + fmaf(a2, tc, c.sig_l2e_lo * t);
  float e2 = ex2_approx(a2);
  e2 = fmaf(e2, kLn2 * a2l, e2);
  const float a3 = c.gsig_l2e * t;
  const float a3l = fmaf(c.gsig_l2e, t, -a3) + fmaf(a3, tc, c.gsig_l2e_lo * t);
  const float e3 = ex2_approx(a3);
  o.e3 = fmaf(e3, kLn2 * a3l, e3);
  const float invr = fmaf(v, ev, v);
  const float t2 = t * t;
  const float t2l = fmaf(t, t, -t2) + 2.0f * t2 * tc;  // t^2 (1 + 2 tc) = t2 + t2l
  o.r = r + dr;
  o.invr = invr;
  o.nde = c.gsig * fmaf(t2, 2.0f * tc, t2);
  const float ae2 = c.Aeps * e2;
  if (c.p == 4 && c.q == 0) {
    // u = sig / r, y = B u^4, each as hi + lo
    const float uh = c.sig * v;
    const float ul = fmaf(c.sig, v, -uh) + fmaf(uh, ev, c.sig_lo * v);
    const float u2 = uh * uh;
    const float u2l = fmaf(uh, uh, -u2) + 2.0f * uh * ul;
    const float u4 = u2 * u2;
    const float u4l = fmaf(u2, u2, -u4) + 2.0f * u2 * u2l;
    const float yh = c.B * u4;
    const float yl = fmaf(c.B, u4, -yh) + fmaf(c.B, u4l, c.B_lo * u4);
    // 1 - y by two-sum (y exceeds 1 only for atoms closer than 2.1 A)
    const float om = 1.0f - yh;
    const float ob = om - 1.0f;
    const float oml = ((1.0f - (om - ob)) + (-yh - ob)) - yl;
    // part 1: (1 - y) sig t^2
    const float qh = c.sig * t2;
    const float ql = fmaf(c.sig, t2, -qh) + fmaf(c.sig, t2l, c.sig_lo * t2);
    const float p1 = om * qh;
    const float p1l = fmaf(om, qh, -p1) + fmaf(om, ql, oml * qh);
    // part 2: -4 y / r
    const float p2 = -4.0f * (yh * v);
    const float p2l = -4.0f * (fmaf(yh, v, -yh * v) + fmaf(yh * v, ev, yl * v));
    // their sum by two-sum, the low parts added once
    const float sh = p1 + p2;
    const float bb = sh - p1;
    const float se = (p1 - (sh - bb)) + (p2 - bb);
    const float g = sh + (se + p1l + p2l);
    o.dphi = ae2 * g;
    o.phi = -ae2 * (om + oml);
  } else {
    const float sr = c.sig * invr;
    const float srp = powi(sr, c.p), srq = powi(sr, c.q);
    const float brk = fmaf(c.B, srp, -srq);
    o.phi = ae2 * brk;
    o.dphi = ae2 * (fmaf((float)(-c.p) * c.B, srp, (float)c.q * srq) * invr - brk * c.sig * fmaf(t2, 2.0f * tc, t2));
  }
  return true;
}

__device__ __forceinline__ int cell_of(const uint4& q, const Box& bx) {
  const int cx = (int)(((unsigned long long)q.x * (unsigned)bx.nc[0]) >> 32);
  const int cy = (int)(((unsigned long long)q.y * (unsigned)bx.nc[1]) >> 32);
  const int cz = (int)(((unsigned long long)q.z * (unsigned)bx.nc[2]) >> 32);
  return bx.cell_off + cx + bx.nc[0] * (cy + bx.nc[1] * cz);
}

__device__ __forceinline__ void set_status(Global* g, int st) { atomicCAS(&g->status, 0, st); }

// Arrival on a block counter, acq_rel at gpu scope: after a __syncthreads it
// publishes the whole block's writes (the barrier orders them before thread
// 0's release) and, for the last block to arrive, acquires every other
// block's.  Returns the count including this arrival.
__device__ __forceinline__ unsigned bar_arrive(unsigned* p) {
  unsigned old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(old) : "l"(p) : "memory");
  return old + 1u;
}
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Rebuilds are per box.  On a rebuild step every atom is binned and the scan
// over all cells gives absolute cell starts (every box's counts add up to its
// atom range), but only boxes whose flag kick1 raised (or that the host
// flagged) are re-sorted and re-listed; the others keep their order and list
// and never read their recomputed starts.
__device__ __forceinline__ bool box_flagged(const Dev& d, int b) { return d.bst[b].rebuild != 0; }

// Per-box accumulation of NV values held as FP32 by each thread; the sums
// across blocks are FP64.  Every thread of the block calls it (b < 0 for
// threads without a contribution, whose values must be 0); thread 0 must hold
// the block's first box.  Atoms are box-major, so box ids along a warp are
// non-decreasing.  A warp within one box (nearly all) reduces its NV values
// by a transpose-reduce butterfly (about NV + 5 shuffles in all); a warp that
// straddles boxes runs a segmented FP32 scan over each run of one box.  Sums
// of the block's first and last box are combined in shared memory (FP32) and
// widened to FP64 for one global atomic per value and block; sums of other
// boxes (small boxes only) go to global memory directly.
template <int NV, class Dst>
__device__ void box_accumulate(float (&v)[NV], int b, Dst dst) {
  static_assert(NV <= 16, "two slots of NV sums are flushed by warp 0");
  __shared__ float sacc[2][NV];
  __shared__ int sbox[2];
  const int lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    sbox[0] = b;
    sbox[1] = -1;
  }
  if (threadIdx.x < 2 * NV) (&sacc[0][0])[threadIdx.x] = 0.f;
  __syncthreads();
  if (b >= 0) atomicMax(&sbox[1], b);  // the block's last box (box ids never decrease along atoms)
  const int b0 = __shfl_sync(kFull, b, 0);
  constexpr bool kPow2 = (NV & (NV - 1)) == 0;
  if (kPow2 && __all_sync(kFull, b == b0 || b < 0)) {
    // the warp holds one box (the common case): transpose-reduce, each of the
    // NV sums ending on its own group of 32/NV lanes
    int off = 16;
#pragma unroll
    for (int n = NV; n > 1; n >>= 1) {
      const bool up = (lane & off) != 0;
#pragma unroll
      for (int k = 0; k < n / 2; ++k) {
        const float send = up ? v[k] : v[k + n / 2];
        const float keep = up ? v[k + n / 2] : v[k];
        v[k] = keep + __shfl_xor_sync(kFull, send, off);
      }
      off >>= 1;
    }
#pragma unroll
    for (; off > 0; off >>= 1) v[0] += __shfl_xor_sync(kFull, v[0], off);
    __syncthreads();
    constexpr int kGroup = 32 / NV;
    if (b0 >= 0 && lane % kGroup == 0) {
      const int k = lane / kGroup;
      const int slot = (b0 == sbox[0]) ? 0 : ((b0 == sbox[1]) ? 1 : -1);
      if (slot >= 0) atomicAdd(&sacc[slot][k], v[0]);
      else atomicAdd(dst(b0) + k, (double)v[0]);
    }
  } else {
    // segmented FP32 scan over the runs of one box in the warp
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int bo = __shfl_up_sync(kFull, b, off);
#pragma unroll
      for (int k = 0; k < NV; ++k) {
        const float vo = __shfl_up_sync(kFull, v[k], off);
        if (lane >= off && bo == b) v[k] += vo;
      }
    }
    const int bn = __shfl_down_sync(kFull, b, 1);
    __syncthreads();
    const bool tail = (b >= 0) && (lane == 31 || bn != b);
    if (tail) {
      const int slot = (b == sbox[0]) ? 0 : ((b == sbox[1]) ? 1 : -1);
      if (slot >= 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) atomicAdd(&sacc[slot][k], v[k]);
      } else {
        double* p = dst(b);
#pragma unroll
        for (int k = 0; k < NV; ++k) atomicAdd(p + k, (double)v[k]);
      }
    }
  }
  __syncthreads();
  // warp 0 alone reads the shared sums after the barrier, so a following call
  // (whose warp 0 resets them first) cannot race with these reads
  if (threadIdx.x < NV && sbox[0] >= 0) atomicAdd(dst(sbox[0]) + threadIdx.x, (double)sacc[0][threadIdx.x]);
  if (threadIdx.x >= 16 && threadIdx.x < 16 + NV && sbox[1] >= 0 && sbox[1] != sbox[0])
    atomicAdd(dst(sbox[1]) + (threadIdx.x - 16), (double)sacc[1][threadIdx.x - 16]);
}

// ---------------------------------------------------------------------------
// Thermostat (Sec. II.B: Nose-Hoover, tau = 1 ps; Berendsen as the option).
// GB300 issues an FP64 instruction at a small fraction of the FP32 rate, even
// for one active lane, so the per-step thermostat arithmetic is FP32: xi and
// eta are unevaluated FP32 pairs hi + lo (their increments are tiny against
// their values), the kinetic energy enters through d = 2 KE - N_df k_B T0,
// formed with one FP64 FMA from the FP64 sum, and a velocity scale s is
// carried as sig = s - 1 (expm1f): the kick applies v += sig v, and the
// relative FP32 error of sig (~1e-4 in size) is ~1e-12 of s.

// a += b for an unevaluated pair a = (hi, lo) and an FP32 b (two-sum).
__device__ __forceinline__ void df_add(float& hi, float& lo, float b) {
  const float s = hi + b;
  const float bb = s - hi;
  const float e = (hi - (s - bb)) + (b - bb);
  const float l = lo + e;
  hi = s + l;
  lo = l - (hi - s);
}

struct ThermoState {  // one box at a step boundary
  float xh, xl, eh, el;  // xi, eta as hi + lo
  float d;               // 2 KE - N_df k_B T0 (FP32)
  float ke;              // KE in FP32 (for the scale's effect on d)
};

// One Nose-Hoover half step (length dt/2) of a single thermostat: quarter step
// on xi, velocity scale exp(-xi dt/2), half step on eta, quarter step on xi.
// Returns sig = s - 1; KE and d follow the scale.
__device__ __forceinline__ float nh_half(const Integ& I, const Box& bx, ThermoState& t) {
  const float hdt = 0.5f * (float)I.dt;
  df_add(t.xh, t.xl, bx.q4f * t.d);
  const float sig = expm1f(-hdt * t.xh);
  const float f = sig * (2.0f + sig);  // s^2 - 1
  const float dke = t.ke * f;
  t.ke += dke;
  t.d = fmaf(2.0f, dke, t.d);
  df_add(t.eh, t.el, hdt * t.xh);
  df_add(t.xh, t.xl, bx.q4f * t.d);
  return sig;
}

// End-of-step half, after the second half-kick: Nose-Hoover half step, or
// the Berendsen scale s = sqrt(1 + dt/tau (T0/T - 1)) (sig = x / (s + 1) with
// x = dt/tau (T0/T - 1), free of cancellation); NVE changes nothing.
// (kNpt: the isobaric instantiation, whose thermostat is always Nose-Hoover)
template <bool kNpt = false>
__device__ __forceinline__ float end_half(const Integ& I, const Box& bx, ThermoState& t) {
  if (kNpt || I.kind == TH_NH) return nh_half(I, bx, t);
  if (I.kind == TH_BERENDSEN && t.ke > 0.f) {
    const float T = 2.0f * t.ke * (float)bx.inv_ndf_kb;
    const float x = (float)(I.dt / I.tau) * ((float)bx.T0 / T - 1.0f);
    const float sig = x / (sqrtf(1.0f + x) + 1.0f);
    const float f = sig * (2.0f + sig);
    t.ke += t.ke * f;
    return sig;
  }
  return 0.f;
}

// Start-of-step half, before the first half-kick (Nose-Hoover only).
template <bool kNpt = false>
__device__ __forceinline__ float start_half(const Integ& I, const Box& bx, ThermoState& t) {
  return (kNpt || I.kind == TH_NH) ? nh_half(I, bx, t) : 0.f;
}

__device__ __forceinline__ ThermoState thermo_in(const Box& bx, float4 th, double ke) {
  ThermoState t;
  t.xh = th.x;
  t.xl = th.y;
  t.eh = th.z;
  t.el = th.w;
  t.d = (float)fma(2.0, ke, -bx.ndfkT0);
  t.ke = (float)ke;
  return t;
}

// Thermo record of box b for the last completed step (parity pp): the
// thermostat state after its end half and the step's energies and virial.
// Written only when the host reads it (k_record).
__device__ void write_record(const Dev& d, const Integ& I, int b, int pp, unsigned long long step_done) {
  const BoxState* st = d.bst + b;
  const Box& bx = d.box[b];
  double* r = d.thermo + (size_t)b * TR_N;
  const double e2 = st->ew[pp][0], e3 = st->ew[pp][1];
  const double ke = st->ke_last;
  const double xi = (double)st->th_e.x + (double)st->th_e.y, eta = (double)st->th_e.z + (double)st->th_e.w;
  const double V = bx.volume;  // the box of the completed step (the next one is made current in its kick1)
  r[TR_STEP] = (double)step_done;
  r[TR_PE] = e2 + e3;
  r[TR_E2] = e2;
  r[TR_E3] = e3;
  r[TR_KE] = ke;
  r[TR_T] = 2.0 * ke * bx.inv_ndf_kb;
  double cons = ke + e2 + e3;
  if (I.kind == TH_NH || I.kind == TH_NPT) cons += 0.5 * bx.Q * xi * xi + bx.ndfkT0 * eta;
  if (I.kind == TH_NPT) cons += I.p_ext * V + 0.5 * st->pe_e * st->pe_e / bx.W;
  r[TR_CONS] = cons;
  r[TR_P] = (2.0 * ke + st->ew[pp][2] + st->ew[pp][3] + st->ew[pp][4]) / (3.0 * V) * kATM;
  for (int k = 0; k < 6; ++k) r[TR_W0 + k] = st->ew[pp][2 + k];
  r[TR_XI] = xi;
  r[TR_ETA] = eta;
  r[TR_REBUILDS] = (double)st->rebuilds;
  r[TR_VOL] = V;
  for (int k = 0; k < 3; ++k) r[TR_L0 + k] = bx.L[k];
}

// Isotropic barostat (Sec. II.B, read as the Martyna-Tobias-Klein form):
// half step on its momentum, pe += dt/2 [(1 + 3/N_df) 2 KE + tr(W) - 3 P V],
// and the friction on the velocities, v *= exp(-dt/2 (1 + 3/N_df) pe/W),
// returned as s - 1 (FP32).  pe and the volume stay FP64.  The geometry is
// read with L2 loads (__ldcg): in the persistent engine another block wrote
// it earlier in the same launch.
__device__ __forceinline__ void baro_half(const Integ& I, const Box& bx, double ke, double trw, double& pe) {
  pe += 0.5 * I.dt * (bx.a3 * 2.0 * ke + trw - 3.0 * I.p_ext * __ldcg(&bx.volume));
}
__device__ __forceinline__ float baro_friction(const Integ& I, const Box& bx, double pe) {
  return expm1f((float)(-0.5 * I.dt * bx.a3 * pe / bx.W));
}

// The box of the coming step: every edge scaled by e^u, u = dt pe/W, during
// its drift.  A box fraction then advances by (v dt / L) (1 - e^-u)/u (the
// drift r -> r e^u + v dt e^(u/2) sinh(u/2)/(u/2) divided by the new edge),
// which the kick kernel's drift factor absorbs; the new edges (Ln) become
// current after that drift, in time for the list build and the force.
// Rebuild margin: a pair outside the list (r >= r_list at the build) is at
// least c r_list - 2 d apart, c = L/L_build, d the largest displacement
// since the build, so the list holds while 2 d <= r_list - r_c -
// r_list max(0, 1 - c); the displacement is measured with the current
// edges, e^-u of the new ones.  A margin below skin/2 rebuilds at once.
__device__ void npt_geometry(const Dev& d, const Integ& I, int b, double pe) {
  Box& bx = const_cast<Box*>(d.box)[b];
  BoxState* st = d.bst + b;
  const float u = (float)(I.dt * pe / bx.W);
  const float eu = expm1f(u);
  const float fdr = fabsf(u) > 1e-3f ? -expm1f(-u) / u : fmaf(u, fmaf(u, 1.0f / 6.0f, -0.5f), 1.0f);
  const float dt64 = (float)(I.dt * 18446744073709551616.0);  // dt 2^64
  bool grid = false;
  for (int k = 0; k < 3; ++k) {
    const double L = __ldcg(&bx.L[k]);
    const double Ln = fma(L, (double)eu, L);
    bx.dtL64[k] = dt64 / (float)L * fdr;
    bx.Ln[k] = Ln;
    const int nc = bx.nc[k];
    if (Ln < 2.0 * I.rlist || (nc >= 4 && Ln < nc * (double)I.rlist) || Ln >= (nc + 1) * kCellGrow * I.rlist)
      grid = true;
  }
  if (grid) set_status(d.g, ST_GRID);
  const float c = (float)(bx.Ln[0] / __ldcg(&st->Lb));
  const float m = I.skin - I.rlist * fmaxf(0.0f, 1.0f - c);
  if (m < 0.5f * I.skin) {
    st->rebuild = 1;
    d.g->any_rebuild = 1;
  }
  const float h = 0.5f * fmaxf(m, 0.0f) / (1.0f + eu);
  bx.hs2 = h * h;
}

// The edges of the coming step made current (the last block of kick1, once
// every block has drifted with the old ones).
__device__ void npt_commit_box(const Dev& d, int b) {
  Box& bx = const_cast<Box*>(d.box)[b];
  double vol = 1.0;
  for (int k = 0; k < 3; ++k) {
    const double Ln = __ldcg(&bx.Ln[k]);
    bx.L[k] = Ln;
    bx.Lq[k] = (float)(Ln * 2.3283064365386963e-10);  // 2^-32
    bx.qs[k] = 4294967296.0 / Ln;
    vol *= Ln;
  }
  bx.volume = vol;
  bx.p_fac = kATM / (3.0 * vol);
}

// Isobaric end-of-step tail (kNpt instantiations only, so that the FP64
// barostat arithmetic does not raise the register count of the others).
__device__ void end_of_step_box_npt(const Dev& d, const Integ& I, int b, int par) {
  BoxState* st = d.bst + b;
  const Box& bx = d.box[b];
  const double ke0 = __ldcg(&st->ke_acc[par]);
  // end of this step: friction, barostat half, thermostat half; start of
  // the next: thermostat half, barostat half, friction; then the new box
  const double trw = __ldcg(&st->ew[par][2]) + __ldcg(&st->ew[par][3]) + __ldcg(&st->ew[par][4]);
  double pe = __ldcg(&st->pe_b);
  const float f1 = baro_friction(I, bx, pe);
  double ke = fma(ke0, (double)(f1 * (2.0f + f1)), ke0);
  baro_half(I, bx, ke, trw, pe);
  ThermoState t = thermo_in(bx, __ldcg(&st->th), ke);
  const float se = end_half<true>(I, bx, t);
  ke = fma(ke, (double)(se * (2.0f + se)), ke);
  st->th_e = make_float4(t.xh, t.xl, t.eh, t.el);
  st->ke_last = ke;
  st->pe_e = pe;
  const float e1 = fmaf(f1, se, f1 + se);
  st->s_endc = 1.0 + (double)e1;
  const float ss = start_half<true>(I, bx, t);
  ke = fma(ke, (double)(ss * (2.0f + ss)), ke);
  st->th = make_float4(t.xh, t.xl, t.eh, t.el);
  baro_half(I, bx, ke, trw, pe);
  const float f2 = baro_friction(I, bx, pe);
  const float e2 = fmaf(ss, f2, ss + f2);
  st->sig = fmaf(e1, e2, e1 + e2);
  st->pe_b = pe;
  npt_geometry(d, I, b, pe);
}

// Thermostat at the end of the step of parity par, for box b (one thread per
// box, after the step's kinetic-energy sum is complete): the end half of this
// step, then the start half of the next one; stores the state after each half
// and the combined scale S - 1 the next kick1 applies.
template <bool kNpt>
__device__ void end_of_step_box(const Dev& d, const Integ& I, int b, int par) {
  if constexpr (kNpt) {
    end_of_step_box_npt(d, I, b, par);
  } else {
    BoxState* st = d.bst + b;
    const Box& bx = d.box[b];
    const double ke0 = __ldcg(&st->ke_acc[par]);
    ThermoState t = thermo_in(bx, __ldcg(&st->th), ke0);
    const float se = end_half(I, bx, t);
    st->th_e = make_float4(t.xh, t.xl, t.eh, t.el);
    st->ke_last = fma(ke0, (double)(se * (2.0f + se)), ke0);
    st->s_endc = 1.0 + (double)se;
    const float ss = start_half(I, bx, t);
    st->th = make_float4(t.xh, t.xl, t.eh, t.el);
    st->sig = fmaf(se, ss, se + ss);
  }
}

// Start half only, from the state after the last end half (a new state, or a
// changed integrator): the scale S - 1 includes the pending end scale.
__global__ void k_prime_thermostat(Dev d) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= d.nbox) return;
  const Integ I = *d.integ;
  BoxState* st = d.bst + b;
  const Box& bx = d.box[b];
  ThermoState t = thermo_in(bx, st->th_e, st->ke_last);
  const float se = (float)(st->s_endc - 1.0);
  const float ss = I.kind == TH_NPT ? start_half<true>(I, bx, t) : start_half(I, bx, t);
  st->th = make_float4(t.xh, t.xl, t.eh, t.el);
  float e2 = ss;
  if (I.kind == TH_NPT) {  // barostat half and friction with the latest virial
    const int wp = d.g->wpar;
    const double trw = st->ew[wp][2] + st->ew[wp][3] + st->ew[wp][4];
    const double ke = fma(st->ke_last, (double)(ss * (2.0f + ss)), st->ke_last);
    double pe = st->pe_e;
    baro_half(I, bx, ke, trw, pe);
    const float f2 = baro_friction(I, bx, pe);
    e2 = fmaf(ss, f2, ss + f2);
    st->pe_b = pe;
    npt_geometry(d, I, b, pe);
  }
  st->sig = fmaf(se, e2, se + e2);
}

// Uniform early exit of a block on a device error status (one read, shared),
// so that no warp skips a barrier the others wait at.
__device__ __forceinline__ bool block_stop(const Dev& d) {
  __shared__ int s_stop;
  if (threadIdx.x == 0) s_stop = *(volatile int*)&d.g->status;
  __syncthreads();
  return s_stop != 0;
}

// ---------------------------------------------------------------------------
// Phase bodies (one item each) shared by the per-phase kernels and the
// persistent kernel.

// a1 + a7 (first half): the second half-kick of the last step and the first
// of this one use the same force, so they are folded: v = S v + (S + 1) a
// when a half-kick is pending (S = thermostat scale of the step boundary,
// a = dt/2 F/m), else v = S v + a; then s += (dt/L) v on the box fraction,
// fixed-point copy, displacement check against the last build.  One thread
// per atom, its three components in turn: every array is read and written
// with one coalesced vector access per warp (the force and the fixed-point
// copies as 16-byte records, the velocity and fraction components as 8-byte
// words), and the box's constants are loaded once per atom.  No FP64
// instruction: v is the unevaluated sum hi + lo of two FP32 values, updated
// as hi + t with t = (S - 1) v + kick and the rounding error of that sum
// carried into lo (Knuth's two-sum); the drift (dt/L) v 2^64 is rounded once
// to FP32 and added exactly to the 64-bit box fraction, which wraps at the
// faces by itself.  The runaway check is an integer test of the FP32
// exponent.  Also zeroes f for this step.
constexpr int kKThreads = 256;  // threads per block of k_kick1 / k_kick2

template <bool kNpt>
__device__ __forceinline__ void kick1_atom(const Dev& d, const Integ& I, int i, int par, int pend) {
  // every load first (nothing here is written by another atom's thread);
  // the fixed-point copy is read only for its box (one box: box 0)
  const int b = d.nbox == 1 ? 0 : (int)d.q[i].w;
  const float4 F = d.f[i];
  const uint4 qb = d.qb[i];
  const float2 v0[3] = {d.vx[i], d.vy[i], d.vz[i]};
  const unsigned long long s0[3] = {d.x[i], d.y[i], d.z[i]};
  const Box& bx = d.box[b];
  const float sig = d.bst[b].sig;
  const float kf = I.cf_f * (pend ? 2.0f + sig : 1.0f);
  const int vexp = bx.vexp_lost;
  const float Fc[3] = {F.x, F.y, F.z};
  const uint32_t qbc[3] = {qb.x, qb.y, qb.z};
  float2 vn[3];
  unsigned long long sn[3];
  uint32_t qn[3];
  float dd = 0.f;  // squared displacement since the last build
  bool lost = false;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    // v + t as hi + lo: two-sum of hi and t, its error added to lo, renormalised
    const float t = fmaf(sig, v0[c].x, fmaf(sig, v0[c].y, kf * Fc[c]));
    const float sh = v0[c].x + t;
    const float bb = sh - v0[c].x;
    const float er = (v0[c].x - (sh - bb)) + (t - bb);
    const float lo1 = v0[c].y + er;
    const float hi = sh + lo1;
    const float lo = lo1 - (hi - sh);
    const float k64 = bx.dtL64[c];
    const long long inc = f2ll_exact(fmaf(hi, k64, lo * k64));
    sn[c] = s0[c] + (unsigned long long)inc;
    if (inc > 0 ? sn[c] < s0[c] : sn[c] > s0[c])  // the 64-bit fraction wrapped: the atom crossed a face
      reinterpret_cast<int*>(d.img + i)[c] += inc > 0 ? 1 : -1;
    vn[c] = make_float2(hi, lo);
    qn[c] = q_of(sn[c]);
    const float dc = fix_diff(qbc[c], qn[c], bx.Lq[c]);
    dd += __fmul_rn(dc, dc);
    // |v| at or above the box's runaway threshold (or NaN/inf): exponent field test
    lost |= (int)((__float_as_uint(hi) >> 23) & 0xffu) >= vexp;
  }
  d.f[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  d.vx[i] = vn[0];
  d.vy[i] = vn[1];
  d.vz[i] = vn[2];
  d.x[i] = sn[0];
  d.y[i] = sn[1];
  d.z[i] = sn[2];
  d.q[i] = make_uint4(qn[0], qn[1], qn[2], (unsigned)b);
  if (i == bx.off) {  // this step's accumulators start from zero
    BoxState* sw = d.bst + b;
    sw->ke_acc[par] = 0.0;
#pragma unroll
    for (int k2 = 0; k2 < 8; ++k2) sw->ew[par][k2] = 0.0;
  }
  if (dd > (kNpt ? bx.hs2 : I.half_skin2)) {
    d.bst[b].rebuild = 1;
    d.g->any_rebuild = 1;
  }
  if (lost) {
    set_status(d.g, ST_LOST);
    d.g->err_index = i;
  }
}

// a7 (second half): the kinetic energy of atom i's v + a (FP32 per
// component and per atom; the sums over atoms are FP64).  The half-kick
// itself is left pending and folded into the next kick1 (or applied when the
// state is read).  b: the atom's box (-1 past the last atom).
__device__ __forceinline__ float kick2_atom(const Dev& d, const Integ& I, int i, int& b) {
  b = -1;
  if (i >= d.N) return 0.f;
  b = d.nbox == 1 ? 0 : (int)d.q[i].w;
  const float4 F = d.f[i];
  const float2 v[3] = {d.vx[i], d.vy[i], d.vz[i]};
  const float Fc[3] = {F.x, F.y, F.z};
  float ke = 0.f;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float u = fmaf(I.cf_f, Fc[c], v[c].x) + v[c].y;
    ke += (float)I.ke_fac * u * u;
  }
  if (!(ke < 1e30f)) {
    set_status(d.g, ST_NAN);
    d.g->err_index = i;
  }
  return ke;
}

// ---------------------------------------------------------------------------
// Neighbour list (a3): one warp per cell.  The candidates of the
// (deduplicated) 27-cell stencil are flattened in stencil order and staged,
// up to kNStage at a time, in the warp's slice of shared memory; then the
// centre atoms of the cell, kNeighCentres at a time, run over the staged
// candidates 32 at a time (one per lane), and the hits of each batch go
// straight to their places in each centre's row (its running count plus the
// hits of lower lanes), so each row lists its neighbours in stencil order.
constexpr int kNStage = 256;  // candidates staged per warp at a time (4 KB)
constexpr int kNeighCentres = 2;  // centres tested together against each staged batch
__device__ __forceinline__ int stencil_n(int nc) { return nc >= 3 ? 3 : nc; }
__device__ __forceinline__ int stencil_off(int nc, int o) { return nc >= 3 ? o - 1 : o; }

// The rows of one cell's centres (neigh_cell_warp).  Staging: lane t of a
// batch takes candidate t of the stencil's concatenated cells (located by a
// binary search over the warp's inclusive counts) and stores (x, y, z, j);
// entries past the last candidate get j = -1 (and, with kFrame, an offset
// no distance test passes).  The centres go over a batch kNeighCentres at a
// time, so that each staged record is read once for all of them (2 measured
// fastest against 1, 3 and 4).  A count past the row
// width (an overflow: the status makes the caller grow the rows and build
// again) writes to the row's last slot, never past it.
// kFrame: every axis of the box has at least 4 cells, so each candidate lies
// within two cell edges of o, the cell's first atom; offsets from o are exact
// fixed-point differences with no wrap, converted once per atom and staged
// as FP32, and a pair's displacement is their FP32 difference.  Otherwise
// (grids of 1-3 cells on an axis, where the stencil wraps round the box) the
// fixed-point coordinates are staged and each pair takes its own
// minimum-image fixed-point difference.
template <bool kFrame>
__device__ __forceinline__ void neigh_rows(const Dev& d, const uint4* qa, float4* stg, int a0, int ni, int incl,
                                           int start, int excl, int total, float L0, float L1, float L2, float rl2) {
  const int lane = threadIdx.x & 31;
  const unsigned below = (1u << lane) - 1u;  // lanes under this one
  const uint4 o = qa[a0];
  for (int ib = 0; ib < ni; ib += 32) {  // centre atoms of this cell, 32 at a time
    const int nb = min(32, ni - ib);
    const int me = a0 + ib + min(lane, nb - 1);  // lane k's centre
    const uint4 qmine = qa[me];
    float cx, cy, cz;  // its offset from o (kFrame) or its fixed-point position
    if constexpr (kFrame) {
      cx = fix_diff(o.x, qmine.x, L0); cy = fix_diff(o.y, qmine.y, L1); cz = fix_diff(o.z, qmine.z, L2);
    } else {
      cx = __uint_as_float(qmine.x); cy = __uint_as_float(qmine.y); cz = __uint_as_float(qmine.z);
    }
    int mycount = 0;  // neighbours of lane k's centre so far
    for (int c0 = 0; c0 < total; c0 += kNStage) {  // chunks of the candidate list (warp-uniform)
      const int nch = min(kNStage, total - c0);
      const int nbat = (nch + 31) >> 5;
      __syncwarp();  // the previous chunk's readers are done
      for (int bt = 0; bt < nbat; ++bt) {
        const int t = c0 + (bt << 5) + lane;
        int lo = 0, hi = 31;
#pragma unroll
        for (int it = 0; it < 5; ++it) {  // smallest lane k with incl_k > t
          const int mid = (lo + hi) >> 1;
          const int v = __shfl_sync(kFull, incl, mid);
          if (v > t) hi = mid; else lo = mid + 1;
        }
        const int sk = __shfl_sync(kFull, start, lo);
        const int ek = __shfl_sync(kFull, excl, lo);
        float4 e = make_float4(kFrame ? 1e30f : 0.f, 0.f, 0.f, __int_as_float(-1));
        if (t < total) {
          const int j = sk + (t - ek);
          const uint4 qj = qa[j];
          if constexpr (kFrame)
            e = make_float4(fix_diff(o.x, qj.x, L0), fix_diff(o.y, qj.y, L1), fix_diff(o.z, qj.z, L2), __int_as_float(j));
          else
            e = make_float4(__uint_as_float(qj.x), __uint_as_float(qj.y), __uint_as_float(qj.z), __int_as_float(j));
        }
        stg[(bt << 5) + lane] = e;
      }
      __syncwarp();
      for (int k = 0; k < nb; k += kNeighCentres) {  // kNeighCentres centres over the staged batch (warp-uniform)
        float xc[kNeighCentres], yc[kNeighCentres], zc[kNeighCentres];
        int ic[kNeighCentres], cc[kNeighCentres];
        int* rc[kNeighCentres];
        bool on[kNeighCentres];  // (a last group may hold fewer centres)
        const int wl = d.W - 1;
#pragma unroll
        for (int c = 0; c < kNeighCentres; ++c) {
          on[c] = k + c < nb;
          const int kc = on[c] ? k + c : k;
          xc[c] = __shfl_sync(kFull, cx, kc);
          yc[c] = __shfl_sync(kFull, cy, kc);
          zc[c] = __shfl_sync(kFull, cz, kc);
          ic[c] = a0 + ib + kc;
          cc[c] = __shfl_sync(kFull, mycount, kc);
          rc[c] = d.nbr + (size_t)ic[c] * d.W;
        }
#pragma unroll 2
        for (int bt = 0; bt < nbat; ++bt) {
          const float4 e = stg[(bt << 5) + lane];
          const int j = __float_as_int(e.w);
          // (kFrame: padding entries fail the distance test by their offset)
          const bool live = kFrame || j >= 0;
#pragma unroll
          for (int c = 0; c < kNeighCentres; ++c) {
            float dx, dy, dz;
            if constexpr (kFrame) {
              dx = e.x - xc[c]; dy = e.y - yc[c]; dz = e.z - zc[c];
            } else {
              dx = fix_diff(__float_as_uint(xc[c]), __float_as_uint(e.x), L0);
              dy = fix_diff(__float_as_uint(yc[c]), __float_as_uint(e.y), L1);
              dz = fix_diff(__float_as_uint(zc[c]), __float_as_uint(e.z), L2);
            }
            const bool p = (c == 0 || on[c]) && live && j != ic[c] && fmaf(dx, dx, fmaf(dy, dy, dz * dz)) < rl2;
            const unsigned bm = __ballot_sync(kFull, p);
            st_if(p, rc[c] + min(cc[c] + __popc(bm & below), wl), j);
            cc[c] += __popc(bm);
          }
        }
#pragma unroll
        for (int c = 0; c < kNeighCentres; ++c)
          if (on[c] && lane == k + c) mycount = cc[c];
      }
    }
    if (lane < nb) d.nbr_cnt[me] = mycount;
    // the longest row: one atomic per warp, and none once the running maximum
    // covers it (rather than one per centre on this one word)
    const int wmax = __reduce_max_sync(kFull, lane < nb ? mycount : 0);
    if (lane == 0 && wmax > *(volatile int*)&d.g->max_count) {
      atomicMax(&d.g->max_count, wmax);
      if (wmax > d.W) set_status(d.g, ST_OVERFLOW);
    }
  }
}

// stg: the warp's kNStage float4 of shared memory.
__device__ void neigh_cell_warp(const Dev& d, const uint4* qa, float4* stg, int c, float rl2) {
  const int lane = threadIdx.x & 31;
  const int a0 = d.cell_start[c];
  const int ni = d.cell_start[c + 1] - a0;
  if (ni == 0 || !box_flagged(d, d.cell_box[c])) return;  // warp-uniform
  const Box& bx = d.box[d.cell_box[c]];
  const int cl = c - bx.cell_off;
  const int cx = cl % bx.nc[0], cy = (cl / bx.nc[0]) % bx.nc[1], cz = cl / (bx.nc[0] * bx.nc[1]);
  const bool frame = bx.nc[0] >= 4 && bx.nc[1] >= 4 && bx.nc[2] >= 4;  // warp-uniform
  int start = 0, cnt = 0;
  int X = -1, Y = 0, Z = 0;  // lane's stencil cell
  if (frame) {  // 3 x 3 x 3 distinct cells; offsets -1, 0, 1 wrap by one compare
    if (lane < 27) {
      X = cx + lane % 3 - 1;
      Y = cy + (lane / 3) % 3 - 1;
      Z = cz + lane / 9 - 1;
      X += X < 0 ? bx.nc[0] : (X >= bx.nc[0] ? -bx.nc[0] : 0);
      Y += Y < 0 ? bx.nc[1] : (Y >= bx.nc[1] ? -bx.nc[1] : 0);
      Z += Z < 0 ? bx.nc[2] : (Z >= bx.nc[2] ? -bx.nc[2] : 0);
    }
  } else {
    const int nx = stencil_n(bx.nc[0]), ny = stencil_n(bx.nc[1]), nz = stencil_n(bx.nc[2]);
    if (lane < nx * ny * nz) {
      const int ox = lane % nx, oy = (lane / nx) % ny, oz = lane / (nx * ny);
      X = (cx + stencil_off(bx.nc[0], ox) + bx.nc[0]) % bx.nc[0];
      Y = (cy + stencil_off(bx.nc[1], oy) + bx.nc[1]) % bx.nc[1];
      Z = (cz + stencil_off(bx.nc[2], oz) + bx.nc[2]) % bx.nc[2];
    }
  }
  if (X >= 0) {
    const int cc = bx.cell_off + X + bx.nc[0] * (Y + bx.nc[1] * Z);
    start = d.cell_start[cc];
    cnt = d.cell_start[cc + 1] - start;
  }
  int incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += t;
  }
  const int excl = incl - cnt;
  const int total = __shfl_sync(kFull, incl, 31);
  const float L0 = bx.Lq[0], L1 = bx.Lq[1], L2 = bx.Lq[2];
  if (frame)
    neigh_rows<true>(d, qa, stg, a0, ni, incl, start, excl, total, L0, L1, L2, rl2);
  else
    neigh_rows<false>(d, qa, stg, a0, ni, incl, start, excl, total, L0, L1, L2, rl2);
}

// ---------------------------------------------------------------------------
// Fused two- + three-body force (k_force).  A block holds kFAtoms centre atoms.
//   leg phase A: kG lanes per centre walk its neighbour row; the pairs with
//     r^2 < (a sig)^2 are compacted (ballot + popc within the lane group) into
//     the centre's row of a padded shared-memory leg table;
//   leg phase B: the leg terms, spread over the group's lanes: the pair term
//     is taken by the owner (half energy, full force on the centre, half
//     virial), and the leg's three-body factors go into the table and into
//     the centre's moments (below);
//   leg phase C: each leg's three-body force from the moments, one
//     red.global.add.v4.f32 to the partner, the reaction kept for the centre;
//   per-box FP64 reduction of E2, E3 and the virial.
// Leg data: u (unit vector i->j), ee = sqrt(lam eps) exp(gam sig/(r - a sig)),
// -1/2 dphi2/dr, nde = gam sig/(r - a sig)^2, r, j (tr = 2/r from r).  With c_jk = u_j.u_k and
// D_jk = c_jk - cos th0 a centre's three-body energy (Sec. II.A) is
//   E3_i = sum_{j<k} ee_j ee_k D_jk^2 = 1/2 sum_j ee_j C_j,
// and the force on leg partner j is
//   F_j = ee_j [ nde_j C_j u_j - tr_j (A_j - B_j u_j) ],
//   A_j = sum_{k!=j} ee_k D_jk u_k,  B_j = sum_{k!=j} ee_k D_jk c_jk,
//   C_j = sum_{k!=j} ee_k D_jk^2.
// Because D_jk is affine in u_j.u_k, the three sums follow exactly from the
// centre's moments S0 = sum_k ee_k, s = sum_k ee_k u_k and the symmetric
// M = sum_k ee_k u_k u_k^T (all legs, k = j included):
//   A_j = M u_j - c0 s - self u_j,  B_j = u_j.M u_j - c0 u_j.s - self c_jj,
//   C_j = u_j.M u_j - 2 c0 u_j.s + c0^2 S0 - self D_jj,
// with c0 = cos th0, c_jj = u_j.u_j, D_jj = c_jj - c0 and self = ee_j D_jj
// (the k = j term taken back out).  This is the same sum reordered: O(n) per
// centre instead of O(n^2) leg pairs.
constexpr int kG = 4;                    // lanes per centre in the leg phase
constexpr int kFThreads = 128;
constexpr int kFAtoms = kFThreads / kG;  // centres per block
constexpr int kWAtoms = 32 / kG;         // centres per warp
constexpr int kLPad = kLMax + 1;         // row pitch (float4) of the adjoint's leg tables
constexpr int kPre = 6;                  // neighbour slots per lane fetched ahead in the leg phase (8 spills at 64 registers)

// The force kernel's shared-memory leg table: a row of kRow float4 records
// per centre (kRow a multiple of 8, i.e. of the 8 bank groups a quarter warp's
// 16-byte accesses spread over).  Leg l of centre a sits at a kRow +
// (l ^ ((a KG) & 7)): the XOR moves the centres that share a quarter warp
// onto disjoint bank groups when their lanes step through legs l = g, g + KG,
// ... together (KG = 2 or 4; with 8 lanes a quarter warp holds one centre).
template <int kRow, int kCent = kFAtoms>
struct LegTableT {
  static_assert(kRow % 8 == 0, "rows must cover whole sets of bank groups");
  float4 ue[kCent * kRow];   // phase A: dx, dy, dz, j (int bits); then ux, uy, uz, ee
  float4 aux[kCent * kRow];  // -1/2 dphi, nde, r, j (int bits)
};
using LegTable = LegTableT<kLMax>;
// Several species: a solute's larger cutoff gives its centres more legs, so
// the species instantiation stages up to 48.
constexpr int kLMaxSp = 48;
using LegTableSp = LegTableT<kLMaxSp>;

// Whole owner contribution (pair terms and three-body terms) of a centre with
// more than kLMax legs (rare): legs in local memory, every unordered leg pair
// once, same arithmetic.  Called by the centre's group leader inside k_force,
// out of line so that its local arrays and registers stay off the common path.
template <bool kCount>
__device__ __noinline__ void force_overflow_item(const Dev& d, const FParams& P, int i, int par) {
  const uint4 qi = d.q[i];
  const int b = (int)qi.w;
  const Box& bx = d.box[b];
  int cnt = d.nbr_cnt[i];
  if (cnt > d.W) cnt = d.W;
  float ux[kMaxLegsOverflow], uy[kMaxLegsOverflow], uz[kMaxLegsOverflow], tr[kMaxLegsOverflow],
      nde[kMaxLegsOverflow], ee[kMaxLegsOverflow], rr[kMaxLegsOverflow];
  float ax[kMaxLegsOverflow], ay[kMaxLegsOverflow], az[kMaxLegsOverflow];
  int jj[kMaxLegsOverflow];
  int nl = 0;
  float e2acc = 0.f, px = 0.f, py = 0.f, pz = 0.f, w[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  for (int s = 0; s < cnt; ++s) {
    const int j = d.nbr[(size_t)i * d.W + s];
    const uint4 qj = d.q[j];
    const float dx = fix_diff(qi.x, qj.x, bx.Lq[0]), dy = fix_diff(qi.y, qj.y, bx.Lq[1]),
                dz = fix_diff(qi.z, qj.z, bx.Lq[2]);
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    if (r2 >= P.rc2) continue;
    LegTerms lt;
    if (!leg_terms(r2, P, lt)) continue;
    if (nl >= kMaxLegsOverflow) {
      set_status(d.g, ST_LEGS);
      d.g->err_index = i;
      return;
    }
    const float invr = lt.invr, r = lt.r;
    ux[nl] = dx * invr;
    uy[nl] = dy * invr;
    uz[nl] = dz * invr;
    tr[nl] = 2.0f * invr;
    nde[nl] = lt.nde;
    ee[nl] = P.sle * lt.e3;
    rr[nl] = r;
    jj[nl] = j;
    ax[nl] = ay[nl] = az[nl] = 0.f;
    {  // pair term, owner computes (half energy, full force on the centre, half virial)
      const float dphi = lt.dphi;
      e2acc = fmaf(0.5f, lt.phi, e2acc);
      px = fmaf(dphi, ux[nl], px);
      py = fmaf(dphi, uy[nl], py);
      pz = fmaf(dphi, uz[nl], pz);
      const float wv = -0.5f * dphi * r;
      w[0] = fmaf(wv * ux[nl], ux[nl], w[0]);
      w[1] = fmaf(wv * uy[nl], uy[nl], w[1]);
      w[2] = fmaf(wv * uz[nl], uz[nl], w[2]);
      w[3] = fmaf(wv * ux[nl], uy[nl], w[3]);
      w[4] = fmaf(wv * ux[nl], uz[nl], w[4]);
      w[5] = fmaf(wv * uy[nl], uz[nl], w[5]);
    }
    ++nl;
  }
  if (kCount) atomicAdd((unsigned long long*)&d.g->ntrip, (unsigned long long)(nl * (nl - 1) / 2));
  float e3acc = 0.f;
  for (int j = 0; j < nl; ++j)
    for (int k = j + 1; k < nl; ++k) {
      const float c = fmaf(ux[j], ux[k], fmaf(uy[j], uy[k], uz[j] * uz[k]));
      const float D = c - P.c0;
      const float g = ee[j] * ee[k] * D;
      e3acc = fmaf(g, D, e3acc);
      const float aj = g * tr[j], bj = g * fmaf(c, tr[j], D * nde[j]);
      ax[j] = fmaf(-aj, ux[k], fmaf(bj, ux[j], ax[j]));
      ay[j] = fmaf(-aj, uy[k], fmaf(bj, uy[j], ay[j]));
      az[j] = fmaf(-aj, uz[k], fmaf(bj, uz[j], az[j]));
      const float ak = g * tr[k], bk = g * fmaf(c, tr[k], D * nde[k]);
      ax[k] = fmaf(-ak, ux[j], fmaf(bk, ux[k], ax[k]));
      ay[k] = fmaf(-ak, uy[j], fmaf(bk, uy[k], ay[k]));
      az[k] = fmaf(-ak, uz[j], fmaf(bk, uz[k], az[k]));
    }
  float fx = 0.f, fy = 0.f, fz = 0.f;
  for (int k = 0; k < nl; ++k) {
    red_add_v4(d.f + jj[k], ax[k], ay[k], az[k]);
    fx -= ax[k];
    fy -= ay[k];
    fz -= az[k];
    const float rx = rr[k] * ux[k], ry = rr[k] * uy[k], rz = rr[k] * uz[k];
    w[0] = fmaf(rx, ax[k], w[0]);
    w[1] = fmaf(ry, ay[k], w[1]);
    w[2] = fmaf(rz, az[k], w[2]);
    w[3] = fmaf(rx, ay[k], w[3]);
    w[4] = fmaf(rx, az[k], w[4]);
    w[5] = fmaf(ry, az[k], w[5]);
  }
  red_add_v4(d.f + i, fx + px, fy + py, fz + pz);
  double* p = &d.bst[b].ew[par][0];  // rare path: per-thread FP64 atomics
  atomicAdd(p + 0, (double)e2acc);
  atomicAdd(p + 1, (double)e3acc);
  for (int k = 0; k < 6; ++k) atomicAdd(p + 2 + k, (double)w[k]);
}

template <bool kCount>
__device__ __noinline__ int species_item(const Dev& d, const SpPair* sp, const float2* st, int nsp, int i,
                                         float (&acc)[8]);

// One block of kFAtoms centres (atoms blk*kFAtoms ...); every thread of the
// block calls it.  kSp = 0: one species.  kSp = 1: several species whose
// three-body strengths factor into leg weights (SpPair::h) and whose
// cos theta0 is the centre's (SpPair::c0); every leg carries its own pair
// constants and weight and the moments stay exact.  kSp = 2: any table;
// phase C then walks the leg pairs, each lane its own legs j against every
// other leg k of the centre (each triplet seen from both legs, each visit
// giving the force on its own leg), with lambda epsilon and cos theta0 of
// (centre; j, k) from the shared triplet table stt.  sps is the nsp^2 pair
// table in shared memory; phase A tests each candidate against its own
// pair's cutoff.
// kOwn (one species only): 0 the scatter kernel; 1 and 2 the two passes of
// owner-computes.  Pass 1 takes the legs, the pair terms (energy, force on
// the centre, virial) and each centre's moments, and stores the moments and
// the staged legs per atom.  Pass 2 recomputes the leg terms from the stored
// legs and gives each centre the three-body reaction of its own terms and
// the forces its neighbours' terms put on it (from their stored moments,
// with the leg reversed), so no leg force is scattered; centres over the
// staged-leg limit keep the scatter path (pass 1), and their neighbours add
// their own terms' forces to them by scatter.
template <bool kCount, int kSp = 0, int KG = kG, int kOwn = 0>
__device__ void force_block(const Dev& d, const FParams& P,
                            LegTableT<(kSp ? kLMaxSp : kLMax), kFThreads / KG>& T, int blk, int par,
                            const SpPair* sps = nullptr, int nsp = 1, const float2* stt = nullptr) {
  constexpr int kLM = kSp ? kLMaxSp : kLMax;  // legs staged per centre
  const int lane = threadIdx.x & 31;
  const int g = threadIdx.x & (KG - 1);
  const int a = threadIdx.x / KG;
  const int sw = (a * KG) & 7;                                  // the row's bank-group swizzle
  auto at = [&](int l) { return a * kLM + (l ^ sw); };          // leg l of this centre
  const int i = blk * (kFThreads / KG) + a;
  const bool valid = i < d.N;
  float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // E2, E3, W xx yy zz xy xz yz
  float fx = 0.f, fy = 0.f, fz = 0.f;  // force on the centre (pair part and three-body reaction)
  uint4 qi = make_uint4(0u, 0u, 0u, 0u);
  int cnt = 0, b = -1;
  float L0 = 0.f, L1 = 0.f, L2 = 0.f;
  const SpPair* spi = nullptr;  // the centre's row of the pair table (kSp)
  int ti = 0;                   // the centre's species (kSp)
  if (valid) {
    qi = d.q[i];
    b = (int)qi.w;
    cnt = min(d.nbr_cnt[i], d.W);
    const Box& bx = d.box[b];
    L0 = bx.Lq[0];
    L1 = bx.Lq[1];
    L2 = bx.Lq[2];
    if constexpr (kSp != 0) {
      ti = d.typ[i];
      spi = sps + ti * nsp;
    }
  }
  // ---- leg phase A: row entries and candidate positions are fetched for
  // kPre slots per lane before any is used (two memory latencies per batch
  // instead of a dependent chain per slot).  Distance test only; hits are
  // compacted (ballot + popc in the lane group) into the centre's row as one
  // record (d, j) (several species: (d, r^2) and (species, j)).
  const int iters = __reduce_max_sync(kFull, (cnt + KG - 1) / KG);
  const unsigned gsh = lane & ~(KG - 1);
  const int* row = d.nbr + (size_t)(valid ? i : 0) * d.W;
  int nl = 0;
  // (kSp: the partner's species rides in the record's x slot until phase B)
  auto test_slot = [&](int j, uint32_t jx, uint32_t jy, uint32_t jz, int tj, bool have) {
    bool hit = false;
    float dx = 0.f, dy = 0.f, dz = 0.f, r2 = 0.f;
    if (have) {
      dx = fix_diff(qi.x, jx, L0);
      dy = fix_diff(qi.y, jy, L1);
      dz = fix_diff(qi.z, jz, L2);
      r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
      if constexpr (kSp)
        hit = r2 < spi[tj].rc2;
      else
        hit = r2 < P.rc2;
    }
    const unsigned m = (__ballot_sync(kFull, hit) >> gsh) & ((1u << KG) - 1u);
    const int pos = nl + __popc(m & ((1u << g) - 1u));
    if (hit && pos < kLM) {
      if constexpr (kSp) {  // (the pair's cutoff test needs r^2 again in phase B: kept)
        T.ue[at(pos)] = make_float4(dx, dy, dz, r2);
        T.aux[at(pos)] = make_float4(__int_as_float(tj), 0.f, 0.f, __int_as_float(j));
      } else {  // one record: r^2 is recomputed from d in phase B by the same expression
        T.ue[at(pos)] = make_float4(dx, dy, dz, __int_as_float(j));
      }
    }
    nl += __popc(m);
  };
  if constexpr (kOwn == 2) {  // the legs pass 1 staged, their vectors recomputed
    const int nlg = valid ? d.nleg[i] : 0;
    nl = nlg < 0 ? 0 : nlg;
    for (int l = g; l < nl; l += KG) {
      const int j = d.legs[(size_t)i * kLMax + l];
      const uint4 qj = d.q[j];
      const float dx = fix_diff(qi.x, qj.x, L0), dy = fix_diff(qi.y, qj.y, L1), dz = fix_diff(qi.z, qj.z, L2);
      T.ue[at(l)] = make_float4(dx, dy, dz, __int_as_float(j));
    }
  } else
  // batches of kPre slots per lane, each fetched as a whole (rows, then
  // positions) before its tests: rows longer than KG * kPre cost one more
  // round trip per batch, not per slot
  for (int t0 = 0; t0 < iters; t0 += kPre) {  // warp-uniform
    int jr[kPre];
    uint32_t qx[kPre], qy[kPre], qz[kPre];
    int tj[kPre];
#pragma unroll
    for (int t = 0; t < kPre; ++t) {
      const int s = g + KG * (t0 + t);
      jr[t] = (s < cnt) ? row[s] : -1;
    }
#pragma unroll
    for (int t = 0; t < kPre; ++t) {
      uint4 qj = make_uint4(0u, 0u, 0u, 0u);
      if (jr[t] >= 0) qj = d.q[jr[t]];
      qx[t] = qj.x;
      qy[t] = qj.y;
      qz[t] = qj.z;
      tj[t] = 0;
      if constexpr (kSp)
        if (jr[t] >= 0) tj[t] = d.typ[jr[t]];
    }
    if constexpr (kSp == 0) {
      // one species: every slot's test first, then one compaction per batch
      // (the lane's hits go to the group's running count plus the hits of the
      // group's lower lanes in this batch, in slot order)
      float dx[kPre], dy[kPre], dz[kPre];
      unsigned hits = 0u;  // bit t: slot t is a leg
      int hc = 0;
#pragma unroll
      for (int t = 0; t < kPre; ++t) {
        dx[t] = fix_diff(qi.x, qx[t], L0);
        dy[t] = fix_diff(qi.y, qy[t], L1);
        dz[t] = fix_diff(qi.z, qz[t], L2);
        const bool hit = jr[t] >= 0 && fmaf(dx[t], dx[t], fmaf(dy[t], dy[t], dz[t] * dz[t])) < P.rc2;
        hits |= hit ? 1u << t : 0u;
        hc += hit ? 1 : 0;
      }
      int incl = hc;  // inclusive prefix of the hit counts over the group's lanes
#pragma unroll
      for (int o = 1; o < KG; o <<= 1) {
        const int y = __shfl_up_sync(kFull, incl, o, KG);
        if (g >= o) incl += y;
      }
      int pos = nl + incl - hc;
#pragma unroll
      for (int t = 0; t < kPre; ++t)
        if ((hits >> t) & 1u) {
          if (pos < kLM) T.ue[at(pos)] = make_float4(dx[t], dy[t], dz[t], __int_as_float(jr[t]));
          ++pos;
        }
      nl += __shfl_sync(kFull, incl, lane | (KG - 1));  // the group's hits in this batch
    } else {
#pragma unroll
      for (int t = 0; t < kPre; ++t)
        if (t0 + t < iters) test_slot(jr[t], qx[t], qy[t], qz[t], tj[t], jr[t] >= 0);
    }
  }
  __syncwarp();
  if constexpr (kOwn == 1) {  // the staged legs for pass 2
    for (int l = g; l < min(nl, kLM); l += KG) d.legs[(size_t)i * kLMax + l] = __float_as_int(T.ue[at(l)].w);
    if (valid && g == 0) d.nleg[i] = nl <= kLM ? nl : -1;
  }
  // ---- leg phase B: leg terms for the compacted legs only, spread over the
  // group's lanes: pair term (owner computes), the leg's table entry and its
  // share of the centre's moments S0, s, M.
  const int nstage = (nl <= kLM) ? nl : 0;  // larger centres: force_overflow_item does everything
  float m0 = 0.f, msx = 0.f, msy = 0.f, msz = 0.f;                            // S0, s
  float mxx = 0.f, myy = 0.f, mzz = 0.f, mxy = 0.f, mxz = 0.f, myz = 0.f;     // M
  int nvalid = 0;  // legs inside their own pair's cutoff (kSp counting)
  for (int l = g; l < nstage; l += KG) {
    float4* ue_p = T.ue + at(l);
    float4* ax_p = T.aux + at(l);
    const float4 rec = *ue_p;
    // (one species: the record is d and j; r^2 as in phase A's test)
    const float r2 = kSp ? rec.w : fmaf(rec.x, rec.x, fmaf(rec.y, rec.y, rec.z * rec.z));
    // the leg's terms with the one species' constants, or its pair's (kSp)
    LegTerms lt;
    float p_h = P.sle;
    bool in;
    if constexpr (kSp) {
      const SpPair& pp = spi[__float_as_int(ax_p->x)];
      p_h = kSp == 2 ? 1.0f : pp.h;  // kSp = 2: the strengths come per leg pair in phase C
      in = leg_terms(r2, pp, lt);
    } else {
      in = leg_terms(r2, P, lt);
    }
    if (!in) {  // FP32 rounding put it on the cutoff (or past its pair's): contributes nothing
      *ue_p = make_float4(0.f, 0.f, 0.f, 0.f);
      continue;
    }
    if constexpr (kSp && kCount) ++nvalid;
    const float r = lt.r;
    const float ux = rec.x * lt.invr, uy = rec.y * lt.invr, uz = rec.z * lt.invr;
    const float ee = p_h * lt.e3;
    const float dphi = kOwn == 2 ? 0.f : lt.dphi;  // (pass 2: the pair terms were taken in pass 1)
    if constexpr (kOwn != 2) {
      acc[0] = fmaf(0.5f, lt.phi, acc[0]);
      fx = fmaf(dphi, ux, fx);
      fy = fmaf(dphi, uy, fy);
      fz = fmaf(dphi, uz, fz);
    }
    if constexpr (kOwn == 1) {  // pass 1 has no phase C: the pair virial here
      const float wv = -0.5f * dphi * r;
      acc[2] = fmaf(wv * ux, ux, acc[2]);
      acc[3] = fmaf(wv * uy, uy, acc[3]);
      acc[4] = fmaf(wv * uz, uz, acc[4]);
      acc[5] = fmaf(wv * ux, uy, acc[5]);
      acc[6] = fmaf(wv * ux, uz, acc[6]);
      acc[7] = fmaf(wv * uy, uz, acc[7]);
    }
    if constexpr (kSp == 1) {
      if (p_h == 0.f) {  // no three-body weight (a lambda = 0 pair): its pair virial here, no phase C
        const float wv = -0.5f * dphi * r;
        acc[2] = fmaf(wv * ux, ux, acc[2]);
        acc[3] = fmaf(wv * uy, uy, acc[3]);
        acc[4] = fmaf(wv * uz, uz, acc[4]);
        acc[5] = fmaf(wv * ux, uy, acc[5]);
        acc[6] = fmaf(wv * ux, uz, acc[6]);
        acc[7] = fmaf(wv * uy, uz, acc[7]);
        *ue_p = make_float4(0.f, 0.f, 0.f, 0.f);
        continue;
      }
    }
    *ue_p = make_float4(ux, uy, uz, ee);
    // (-1/2 dphi: the pair term's share of the virial, taken in phase C), nde, r, j
    // (kSp = 2: j with the partner's species in bits 28-30)
    const float jw = kSp == 2 ? __int_as_float(__float_as_int(ax_p->w) | (__float_as_int(ax_p->x) << 28))
                              : (kSp ? ax_p->w : rec.w);
    *ax_p = make_float4(-0.5f * dphi, lt.nde, r, jw);
    if constexpr (kSp == 2) continue;  // no moments
    const float ex = ee * ux, ey = ee * uy, ez = ee * uz;
    m0 += ee;
    msx += ex;
    msy += ey;
    msz += ez;
    mxx = fmaf(ex, ux, mxx);
    myy = fmaf(ey, uy, myy);
    mzz = fmaf(ez, uz, mzz);
    mxy = fmaf(ex, uy, mxy);
    mxz = fmaf(ex, uz, mxz);
    myz = fmaf(ey, uz, myz);
  }
  // the centre's moments: sum over the lane group
#pragma unroll
  for (int o = 1; o < KG; o <<= 1) {
    m0 += __shfl_xor_sync(kFull, m0, o);
    msx += __shfl_xor_sync(kFull, msx, o);
    msy += __shfl_xor_sync(kFull, msy, o);
    msz += __shfl_xor_sync(kFull, msz, o);
    mxx += __shfl_xor_sync(kFull, mxx, o);
    myy += __shfl_xor_sync(kFull, myy, o);
    mzz += __shfl_xor_sync(kFull, mzz, o);
    mxy += __shfl_xor_sync(kFull, mxy, o);
    mxz += __shfl_xor_sync(kFull, mxz, o);
    myz += __shfl_xor_sync(kFull, myz, o);
  }
  __syncwarp();  // the group's table entries are complete
  if constexpr (kOwn == 1) {
    if (valid && g == 0) {
      d.mom[3 * (size_t)i] = make_float4(m0, msx, msy, msz);
      d.mom[3 * (size_t)i + 1] = make_float4(mxx, myy, mzz, mxy);
      d.mom[3 * (size_t)i + 2] = make_float4(mxz, myz, 0.f, 0.f);
    }
  } else if constexpr (kSp == 2) {
    // ---- leg phase C (any table): leg j against every other leg k
    const float2* stc = stt + ti * nsp * nsp;
    for (int l = g; l < nstage; l += KG) {
      const float4 uj = T.ue[at(l)];
      const float4 xj = T.aux[at(l)];
      if (uj.w == 0.f) continue;  // leg dropped in phase B
      const int wj = __float_as_int(xj.w);
      const float2* stj = stc + (wj >> 28) * nsp;
      const float r = xj.z;
      const float tr = 2.0f * rcp_approx(r);
      const float nde = xj.y;
      float gx = 0.f, gy = 0.f, gz = 0.f;  // three-body force on the partner of leg j
      for (int k = 0; k < nstage; ++k) {
        const float4 uk = T.ue[at(k)];
        if (k == l || uk.w == 0.f) continue;
        const float2 lc = stj[__float_as_int(T.aux[at(k)].w) >> 28];  // (lambda eps, cos theta0)
        const float c = fmaf(uj.x, uk.x, fmaf(uj.y, uk.y, uj.z * uk.z));
        const float D = c - lc.y;
        const float gg = lc.x * uj.w * uk.w * D;
        acc[1] = fmaf(0.5f * gg, D, acc[1]);  // each triplet is visited from both of its legs
        const float aj = gg * tr, bj = gg * fmaf(c, tr, D * nde);
        gx = fmaf(-aj, uk.x, fmaf(bj, uj.x, gx));
        gy = fmaf(-aj, uk.y, fmaf(bj, uj.y, gy));
        gz = fmaf(-aj, uk.z, fmaf(bj, uj.z, gz));
      }
      red_add_v4(d.f + (wj & 0x0FFFFFFF), gx, gy, gz);
      fx -= gx;
      fy -= gy;
      fz -= gz;
      const float hx = fmaf(xj.x, uj.x, gx), hy = fmaf(xj.x, uj.y, gy), hz = fmaf(xj.x, uj.z, gz);
      const float rx = r * uj.x, ry = r * uj.y, rz = r * uj.z;
      acc[2] = fmaf(rx, hx, acc[2]);
      acc[3] = fmaf(ry, hy, acc[3]);
      acc[4] = fmaf(rz, hz, acc[4]);
      acc[5] = fmaf(rx, hy, acc[5]);
      acc[6] = fmaf(rx, hz, acc[6]);
      acc[7] = fmaf(ry, hz, acc[7]);
    }
  } else {
  // ---- leg phase C: three-body force on each leg partner from the moments
  const float c0 = (kSp && valid) ? spi[0].c0 : P.c0;
  // a centre with one leg has no three-body term: its moments hold only that
  // leg, whose self term cancels up to rounding; the residue is not computed
  const bool three = nstage > 1;  // (uniform over the centre's lane group)
  // the three-body force on the partner of leg (u, ee, nde, r) of a centre
  // with moments (S0, s, M), and the leg's C; the k = j term is taken back
  // out with c_jj = |u|^2 as computed (not 1), so that it cancels the same
  // product inside the moments
  auto leg_force = [&](float ux, float uy, float uz, float ee, float nde, float r, float S0, float sx, float sy,
                       float sz, float Mxx, float Myy, float Mzz, float Mxy, float Mxz, float Myz, float& gx,
                       float& gy, float& gz) {
    const float mx = fmaf(Mxx, ux, fmaf(Mxy, uy, Mxz * uz));  // M u
    const float my = fmaf(Mxy, ux, fmaf(Myy, uy, Myz * uz));
    const float mz = fmaf(Mxz, ux, fmaf(Myz, uy, Mzz * uz));
    const float qm = fmaf(ux, mx, fmaf(uy, my, uz * mz));     // u.M u
    const float ps = fmaf(ux, sx, fmaf(uy, sy, uz * sz));     // u.s
    const float cjj = fmaf(ux, ux, fmaf(uy, uy, uz * uz));
    const float djj = cjj - c0;
    const float self = ee * djj;
    const float Bj = fmaf(-c0, ps, qm) - self * cjj;
    const float Cj = fmaf(-2.0f * c0, ps, fmaf(c0 * c0, S0, qm)) - self * djj;
    const float Ax = fmaf(-c0, sx, mx) - self * ux;
    const float Ay = fmaf(-c0, sy, my) - self * uy;
    const float Az = fmaf(-c0, sz, mz) - self * uz;
    const float tr = 2.0f * rcp_approx(r);
    const float et = ee * tr;                       // ee_j tr_j
    const float cu = ee * fmaf(nde, Cj, tr * Bj);   // ee_j (nde_j C_j + tr_j B_j)
    gx = fmaf(cu, ux, -et * Ax);
    gy = fmaf(cu, uy, -et * Ay);
    gz = fmaf(cu, uz, -et * Az);
    return Cj;
  };
  for (int l = g; l < nstage; l += KG) {
    const float4 uj = T.ue[at(l)];
    const float4 xj = T.aux[at(l)];
    const float ee = uj.w;
    if (ee == 0.f) continue;  // leg dropped in phase B
    const float r = xj.z;
    const int j = __float_as_int(xj.w);
    float gx = 0.f, gy = 0.f, gz = 0.f;
    if (three) {
      const float Cj = leg_force(uj.x, uj.y, uj.z, ee, xj.y, r, m0, msx, msy, msz, mxx, myy, mzz, mxy, mxz, myz,
                                 gx, gy, gz);
      // the partner's share: scattered (pass 2: gathered by the partner, unless
      // it is a centre over the staged-leg limit)
      if (kOwn == 0 || d.nleg[j] < 0) red_add_v4(d.f + j, gx, gy, gz);
      fx -= gx;
      fy -= gy;
      fz -= gz;
      acc[1] = fmaf(0.5f * ee, Cj, acc[1]);
    }
    if constexpr (kOwn == 2) {  // the partner's terms on this centre, from its moments, leg reversed
      if (d.nleg[j] >= 0) {
        const float4 ma = d.mom[3 * (size_t)j], mb = d.mom[3 * (size_t)j + 1], mc = d.mom[3 * (size_t)j + 2];
        float hx, hy, hz;
        if (d.nleg[j] > 1) {
          leg_force(-uj.x, -uj.y, -uj.z, ee, xj.y, r, ma.x, ma.y, ma.z, ma.w, mb.x, mb.y, mb.z, mb.w, mc.x, mc.y, hx,
                    hy, hz);
          fx += hx;
          fy += hy;
          fz += hz;
        }
      }
    }
    // virial: r u_a (g_b - 1/2 dphi u_b), the three-body and the pair part
    // (pass 2: xj.x = 0, the pair part was taken in pass 1)
    const float hx = fmaf(xj.x, uj.x, gx), hy = fmaf(xj.x, uj.y, gy), hz = fmaf(xj.x, uj.z, gz);
    const float rx = r * uj.x, ry = r * uj.y, rz = r * uj.z;
    acc[2] = fmaf(rx, hx, acc[2]);
    acc[3] = fmaf(ry, hy, acc[3]);
    acc[4] = fmaf(rz, hz, acc[4]);
    acc[5] = fmaf(rx, hy, acc[5]);
    acc[6] = fmaf(rx, hz, acc[6]);
    acc[7] = fmaf(ry, hz, acc[7]);
  }
  }  // phase C
  // ---- force on the centre: pair part + three-body reaction, over the group
#pragma unroll
  for (int o = 1; o < KG; o <<= 1) {
    fx += __shfl_xor_sync(kFull, fx, o);
    fy += __shfl_xor_sync(kFull, fy, o);
    fz += __shfl_xor_sync(kFull, fz, o);
  }
  if (valid && g == 0) {
    red_add_v4(d.f + i, fx, fy, fz);
    if (nl > kLM) {  // rare: more legs than the table holds
      if constexpr (kSp != 0)
        species_item<kCount>(d, sps, d.sp_tri, nsp, i, acc);
      else
        force_overflow_item<kCount>(d, P, i, par);
    }
  }
  if (kCount && kOwn != 2) {  // legs and table-path triplets, one atomic per warp (pass 2 counts nothing)
    int nleg = nl;
    if constexpr (kSp) {  // legs inside their own pair's cutoff, summed over the group
#pragma unroll
      for (int o = 1; o < KG; o <<= 1) nvalid += __shfl_xor_sync(kFull, nvalid, o);
      nleg = nvalid;
    }
    unsigned long long legs = (valid && g == 0 && (!kSp || nl <= kLM)) ? (unsigned long long)nleg : 0ull;
    unsigned long long tri =
        (valid && g == 0 && nl <= kLM) ? (unsigned long long)(nleg * (nleg - 1) / 2) : 0ull;
    for (int o = 16; o > 0; o >>= 1) {
      legs += __shfl_down_sync(kFull, legs, o);
      tri += __shfl_down_sync(kFull, tri, o);
    }
    if (lane == 0) {
      atomicAdd((unsigned long long*)&d.g->npairs, legs);
      atomicAdd((unsigned long long*)&d.g->ntrip, tri);
    }
  }
  box_accumulate<8>(acc, b, [&](int bb) { return &d.bst[bb].ew[par][0]; });
}

// k_force in several launch shapes, picked by the autotuner: KG lanes per
// centre (kFThreads / KG centres per block) and a register budget of MINB
// co-resident blocks per SM (65536 / (kFThreads MINB) registers a thread).
template <bool kCount, int KG = kG, int MINB = 8, int kOwn = 0>
__global__ void __launch_bounds__(kFThreads, MINB) k_force(const __grid_constant__ Dev d, const __grid_constant__ FParams P) {
  if (block_stop(d)) return;
  __shared__ LegTableT<kLMax, kFThreads / KG> T;
  const int par = (int)(d.g->step & 1ull);
  if (blockIdx.x == 0) {  // the rebuild (if any) is consumed
    for (int k = threadIdx.x; k < d.nbox; k += blockDim.x) d.bst[k].rebuild = 0;
    if (threadIdx.x == 0) {
      d.g->any_rebuild = 0;
      d.g->wpar = par;
    }
  }
  force_block<kCount, 0, KG, kOwn>(d, P, T, blockIdx.x, par);
}

// The shapes k_force is built in: {lanes per centre, blocks per SM}.  Shape 0
// is the default; the set spans what a sweep on 2^20 atoms measured within
// 20 % of the best (2 and 8 lanes give more or fewer, larger or smaller
// blocks for small systems).
// Shape 4 is owner-computes (two passes, 4 lanes, 8 blocks per SM) against
// the scatter of the others.
constexpr int kForceShapes = 5;
__host__ __device__ constexpr int force_shape_lanes(int s) { return s == 1 ? 2 : (s == 2 ? 8 : 4); }
__host__ __device__ constexpr int force_shape_blocks(int s) { return s == 3 ? 7 : 8; }
__host__ __device__ constexpr bool force_shape_owner(int s) { return s == 4; }


// ---------------------------------------------------------------------------
// Per-phase kernels (the graph engine and the standalone force call).

// kCond (the graph engine's instantiation): the last block to finish also
// sets the condition of the graph's IF node that holds the rebuild kernels
// (skipped when no box moved more than skin/2).  The other instantiation
// holds no conditional-node call, so profilers can capture it.
// kNpt: the isobaric instantiation (rebuild margin per box, and its last
// block makes the coming step's edges current).
// k_kick1: one atom per thread.  k_kick2: kK2Items atoms per thread, atom
// (blk kK2Items + j) blockDim + t for thread t of block blk (the block's
// threads on consecutive atoms at each j), all loads first; the kinetic
// energies are summed per warp (box by box) and once per block.
constexpr int kK2Items = 4;

// k_kick1 takes a 40-register budget (6 blocks per SM): more loads in flight
// per SM than at its natural 58 registers (26 against 28.5 us at 2^20 atoms).
template <bool kCond, bool kNpt = false>
__global__ void __launch_bounds__(kKThreads, 6) k_kick1(Dev d, cudaGraphConditionalHandle rebuild_cond) {
  if (block_stop(d)) return;
  const Integ I = *d.integ;
  const int par = (int)(d.g->step & 1ull);
  const int pend = d.g->pend;
  if (blockIdx.x == 0 && threadIdx.x == 0) d.g->n_over = 0;
  const int i = (int)(blockIdx.x * blockDim.x + threadIdx.x);
  if (i < d.N) kick1_atom<kNpt>(d, I, i, par, pend);
  if constexpr (kCond || kNpt) {
    __shared__ bool last;
    __syncthreads();
    if (threadIdx.x == 0) last = (bar_arrive(&d.g->done1) == gridDim.x);
    __syncthreads();
    if (last) {
      if constexpr (kNpt)
        for (int b = threadIdx.x; b < d.nbox; b += blockDim.x) npt_commit_box(d, b);
      if (threadIdx.x == 0) {
        d.g->done1 = 0u;
        if constexpr (kCond) cudaGraphSetConditional(rebuild_cond, *(volatile int*)&d.g->any_rebuild ? 1u : 0u);
      }
    }
  }
}

// a2: cell of atom i and its rank among the atoms of that cell (counting sort).
__device__ __forceinline__ void bin_item(const Dev& d, int i) {
  const uint4 q = d.q[i];
  const int c = cell_of(q, d.box[q.w]);
  d.cell[i] = c;
  d.rank[i] = atomicAdd(d.cell_cnt + c, 1);
}

// a2: atom i to its sorted slot in the staging arrays.
__device__ __forceinline__ void scatter_item(const Dev& d, int i) {
  if (!box_flagged(d, (int)d.q[i].w)) return;
  const int p = d.cell_start[d.cell[i]] + d.rank[i];
  if ((unsigned)p >= (unsigned)d.N) {  // counts not cleared after an interrupted build: report, write nothing
    set_status(d.g, ST_CELLS);
    d.g->err_index = i;
    return;
  }
  d.tx[p] = d.x[i]; d.ty[p] = d.y[i]; d.tz[p] = d.z[i];
  d.tvx[p] = d.vx[i]; d.tvy[p] = d.vy[i]; d.tvz[p] = d.vz[i];
  d.tid[p] = d.id[i];
  d.tq[p] = d.q[i];
  d.timg[p] = d.img[i];
  if (d.typ) d.ttyp[p] = d.typ[i];
}

// a2: staging arrays back to the state arrays; build positions recorded.
__device__ __forceinline__ void copyback_item(const Dev& d, int i) {
  if (!box_flagged(d, (int)d.q[i].w)) return;  // a box keeps its atom range
  d.x[i] = d.tx[i]; d.y[i] = d.ty[i]; d.z[i] = d.tz[i];
  d.vx[i] = d.tvx[i]; d.vy[i] = d.tvy[i]; d.vz[i] = d.tvz[i];
  d.id[i] = d.tid[i];
  d.img[i] = d.timg[i];
  if (d.typ) d.typ[i] = d.ttyp[i];
  const uint4 q = d.tq[i];
  d.q[i] = q;
  d.qb[i] = q;
}

__global__ void k_bin(Dev d) {
  if (!d.g->any_rebuild || d.g->status) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) d.g->max_count = 0;
  if (i < d.N) bin_item(d, i);
}

// Exclusive scan of the per-cell counts into cell_start (one block of 1024
// threads, 8 cells per thread per tile), zeroing the counts for the next build.
constexpr int kScanThreads = 1024;
__global__ void __launch_bounds__(kScanThreads) k_scan(Dev d) {
  if (!d.g->any_rebuild || d.g->status) return;
  __shared__ int wsum[32];
  __shared__ int carry_s;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (tid == 0) carry_s = 0;
  __syncthreads();
  constexpr int PER = 8;
  for (int base = 0; base < d.ncell; base += kScanThreads * PER) {
    int v[PER];
    int sum = 0;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int c = base + tid * PER + k;
      v[k] = (c < d.ncell) ? d.cell_cnt[c] : 0;
      sum += v[k];
    }
    int incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    if (wid == 0) {
      int w = wsum[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(kFull, w, o);
        if (lane >= o) w += t;
      }
      wsum[lane] = w;
    }
    __syncthreads();
    int run = carry_s + (wid > 0 ? wsum[wid - 1] : 0) + incl - sum;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int c = base + tid * PER + k;
      if (c < d.ncell) {
        d.cell_start[c] = run;
        d.cell_cnt[c] = 0;
      }
      run += v[k];
    }
    __syncthreads();
    if (tid == 0) carry_s += wsum[31];
    __syncthreads();
  }
  if (tid == 0) d.cell_start[d.ncell] = carry_s;
}

__global__ void k_scatter(Dev d) {
  if (!d.g->any_rebuild || d.g->status) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < d.N) scatter_item(d, i);
}

__global__ void k_copyback(Dev d) {
  if (!d.g->any_rebuild || d.g->status) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) d.g->rebuild_steps += 1;
  if (i < d.nbox && box_flagged(d, i)) {
    d.bst[i].rebuilds += 1;
    d.bst[i].Lb = d.box[i].L[0];
  }
  if (i < d.N) copyback_item(d, i);
}

constexpr int kNeighThreads = 128;
__global__ void __launch_bounds__(kNeighThreads) k_neigh(Dev d, float rl2) {
  if (!d.g->any_rebuild || d.g->status) return;
  __shared__ float4 stg[kNeighThreads / 32][kNStage];
  const int w = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
  if (w < d.ncell) neigh_cell_warp(d, d.q, stg[threadIdx.x >> 5], w, rl2);
}


// a7 second half: kinetic energy of v + a per box; the last block to finish
// runs the thermostat halves of every box (FP32, a short serial tail) and
// advances the step.  The half-kick itself stays pending.
template <bool kNpt = false>
__global__ void __launch_bounds__(kKThreads) k_kick2(Dev d) {
  if (block_stop(d)) return;
  __shared__ float s_ke[kKThreads / 32];
  __shared__ int s_box[kKThreads / 32];
  const Integ I = *d.integ;
  const unsigned long long step = d.g->step;
  const int par = (int)(step & 1ull);
  const int nwb = (int)(blockDim.x >> 5), wib = (int)(threadIdx.x >> 5), lane = (int)(threadIdx.x & 31);
  // per warp: a running FP32 sum for one box; a warp whose item changes box
  // adds its sum to the old box (FP64 atomic) and starts again; an item that
  // itself straddles two boxes is added atom by atom (rare)
  float acc = 0.f;
  int cur = -1;
  float ke[kK2Items];
  int bj[kK2Items];
  {  // every item's loads first, then the arithmetic
    float4 Fj[kK2Items];
    float2 vj[kK2Items][3];
#pragma unroll
    for (int j = 0; j < kK2Items; ++j) {
      const int i = ((int)blockIdx.x * kK2Items + j) * (int)blockDim.x + (int)threadIdx.x;
      const bool act = i < d.N;
      bj[j] = act ? (d.nbox == 1 ? 0 : (int)d.q[i].w) : -1;
      Fj[j] = act ? d.f[i] : make_float4(0.f, 0.f, 0.f, 0.f);
      vj[j][0] = act ? d.vx[i] : make_float2(0.f, 0.f);
      vj[j][1] = act ? d.vy[i] : make_float2(0.f, 0.f);
      vj[j][2] = act ? d.vz[i] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int j = 0; j < kK2Items; ++j) {
      const float Fc[3] = {Fj[j].x, Fj[j].y, Fj[j].z};
      ke[j] = 0.f;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float u = fmaf(I.cf_f, Fc[c], vj[j][c].x) + vj[j][c].y;
        ke[j] += (float)I.ke_fac * u * u;
      }
      if (bj[j] >= 0 && !(ke[j] < 1e30f)) {
        set_status(d.g, ST_NAN);
        d.g->err_index = ((int)blockIdx.x * kK2Items + j) * (int)blockDim.x + (int)threadIdx.x;
      }
    }
  }
#pragma unroll
  for (int j = 0; j < kK2Items; ++j) {
    const int b0 = __shfl_sync(kFull, bj[j], 0);
    if (__all_sync(kFull, bj[j] == b0 || bj[j] < 0)) {
      if (b0 < 0) continue;  // an item past the last atom (warp-uniform)
      float v = ke[j];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
      if (b0 != cur) {
        if (cur >= 0 && lane == 0) atomicAdd(&d.bst[cur].ke_acc[par], (double)acc);
        acc = 0.f;
        cur = b0;
      }
      acc += v;
    } else if (bj[j] >= 0) {
      atomicAdd(&d.bst[bj[j]].ke_acc[par], (double)ke[j]);
    }
  }
  if (lane == 0) {
    s_ke[wib] = acc;
    s_box[wib] = cur;
  }
  __syncthreads();
  if (threadIdx.x == 0) {  // the warps' sums, one FP64 atomic per run of equal boxes
    float run = 0.f;
    int rb = -1;
    for (int w = 0; w < nwb; ++w) {
      if (s_box[w] < 0) continue;
      if (s_box[w] != rb) {
        if (rb >= 0) atomicAdd(&d.bst[rb].ke_acc[par], (double)run);
        run = 0.f;
        rb = s_box[w];
      }
      run += s_ke[w];
    }
    if (rb >= 0) atomicAdd(&d.bst[rb].ke_acc[par], (double)run);
  }
  __shared__ bool am_last;
  if (threadIdx.x == 0) am_last = (bar_arrive(&d.g->done) == gridDim.x);
  __syncthreads();
  if (am_last) {
    for (int bb = threadIdx.x; bb < d.nbox; bb += blockDim.x) end_of_step_box<kNpt>(d, I, bb, par);
    __syncthreads();
    if (threadIdx.x == 0) {
      d.g->done = 0u;
      d.g->pend = 1;
      d.g->step = step + 1ull;
    }
  }
}

__global__ void k_record(Dev d) {
  const Integ I = *d.integ;
  const unsigned long long step = d.g->step;
  const int pl = (int)((step - 1ull) & 1ull);
  for (int b = threadIdx.x; b < d.nbox; b += blockDim.x) write_record(d, I, b, pl, step);
}

// Thermo record from the energies in parity slot pp (a resumed checkpoint).
__global__ void k_record_at(Dev d, int pp) {
  const Integ I = *d.integ;
  const unsigned long long step = d.g->step;
  for (int b = threadIdx.x; b < d.nbox; b += blockDim.x) write_record(d, I, b, pp, step);
}

// ---------------------------------------------------------------------------
// Setup / IO kernels.

// New positions for the current atom order (mw_energy_forces_dev): from a
// user-order AoS device array into the sorted arrays, x[i] = xin[id[i]],
// wrapped into [0, L); q recomputed.
__global__ void k_load_positions(Dev d, const double* __restrict__ xin, const int* __restrict__ boxid) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.N) return;
  const int u = d.id[i];
  const int b = boxid[u];
  const Box& bx = d.box[b];
  unsigned long long p[3];
  int im[3];
  for (int k = 0; k < 3; ++k) {
    double v = xin[3 * (size_t)u + k];
    if (!isfinite(v)) {  // reported to the host, which refuses the state; 0 keeps the arithmetic defined
      set_status(d.g, ST_INPUT);
      d.g->err_index = u;
      v = 0.0;
    }
    v /= bx.L[k];  // box fraction
    const double fl = floor(v);
    im[k] = (int)fl;
    v -= fl;
    if (v >= 1.0) v -= 1.0;
    if (v < 0.0) v = 0.0;
    p[k] = frac64_of(v);
  }
  d.x[i] = p[0]; d.y[i] = p[1]; d.z[i] = p[2];
  if (d.img) d.img[i] = make_int4(im[0], im[1], im[2], 0);
  d.q[i] = make_uint4(q_of(p[0]), q_of(p[1]), q_of(p[2]), (unsigned)b);
}

// Fixed-point copies of restored positions (checkpoint resume): q and the
// build positions qb from the 64-bit fractions, the box from the atom's id.
__global__ void k_requantize(Dev d, const int* __restrict__ boxid) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.N) return;
  const uint4 q = make_uint4(q_of(d.x[i]), q_of(d.y[i]), q_of(d.z[i]), (unsigned)boxid[d.id[i]]);
  d.q[i] = q;
  d.qb[i] = q;
}

// A new state in one pass (mw_set_state): atom i takes the caller's atom i
// (identity order), its species, its velocity (zero when vin is null) and
// zero force, and adds its kinetic energy to its box's ke_last; the cell
// counts are cleared.  The host zeroes the box states and the status block
// before the launch; here each box is marked for a rebuild with no pending
// end scale, and the status block gets the rebuild flag and count_terms.  A
// non-finite value is replaced by 0 and reported (ST_INPUT, the atom in
// err_index); the host refuses the state.
__global__ void k_load_state(Dev d, const double* __restrict__ xin, const double* __restrict__ vin,
                             const int* __restrict__ boxid, int count_terms) {
  const Integ I = *d.integ;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < d.ncell) d.cell_cnt[i] = 0;
  if (i < d.nbox) {
    d.bst[i].s_endc = 1.0;
    d.bst[i].rebuild = 1;
  }
  if (i == 0) {
    d.g->any_rebuild = 1;
    d.g->count_terms = count_terms;
  }
  float ke[1] = {0.f};
  int b = -1;
  if (i < d.N) {
    d.id[i] = i;
    b = boxid[i];
    const Box& bx = d.box[b];
    unsigned long long p[3];
    int im[3];
    float vh[3];
    for (int k = 0; k < 3; ++k) {
      double x = xin[3 * (size_t)i + k];
      if (!isfinite(x)) {
        set_status(d.g, ST_INPUT);
        d.g->err_index = i;
        x = 0.0;
      }
      double f = x / bx.L[k];  // box fraction
      const double fl = floor(f);
      im[k] = (int)fl;
      f -= fl;
      if (f >= 1.0) f -= 1.0;
      if (f < 0.0) f = 0.0;
      p[k] = frac64_of(f);
      double w = vin ? vin[3 * (size_t)i + k] : 0.0;
      if (!isfinite(w)) {
        set_status(d.g, ST_INPUT);
        d.g->err_index = i;
        w = 0.0;
      }
      const float2 sw = split_df(w);
      (k == 0 ? d.vx : (k == 1 ? d.vy : d.vz))[i] = sw;
      vh[k] = sw.x + sw.y;
    }
    d.x[i] = p[0];
    d.y[i] = p[1];
    d.z[i] = p[2];
    if (d.img) d.img[i] = make_int4(im[0], im[1], im[2], 0);
    d.q[i] = make_uint4(q_of(p[0]), q_of(p[1]), q_of(p[2]), (unsigned)b);
    if (d.typ) d.typ[i] = d.utyp[i];
    d.f[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    ke[0] = (float)I.ke_fac * fmaf(vh[0], vh[0], fmaf(vh[1], vh[1], vh[2] * vh[2]));
  }
  box_accumulate<1>(ke, b, [&](int bb) { return &d.bst[bb].ke_last; });
}

// A new state in the current atom order (mw_set_state while that order and
// the neighbour lists are current): sorted slot i takes the caller's atom
// id[i] with the same conversions as k_load_state (positions to 64-bit and
// fixed-point fractions, image counts, velocities as FP32 pairs, species,
// zero force, kinetic energy per box).  A box keeps its list when every one
// of its atoms lies within half the skin (hs2 = (skin/2)^2) of the position
// the list was built at, as between steps; any other box is flagged for a
// rebuild.  The host zeroes the box states and the status block (all but
// the widest-row record) before the launch.
// Per-atom parts of k_load_state_keep: slot i's position (fractions, image
// counts, fixed-point copy, species, zero force, the rebuild flag of its
// box) and its velocity (FP32 pair; returns its kinetic energy).
__device__ __forceinline__ void load_keep_position(const Dev& d, const double* __restrict__ xin, int i, float hs2) {
  const int u = d.id[i];
  const int b = (int)d.q[i].w;
  const Box& bx = d.box[b];
  unsigned long long p[3];
  int im[3];
  for (int k = 0; k < 3; ++k) {
    double x = xin[3 * (size_t)u + k];
    if (!isfinite(x)) {
      set_status(d.g, ST_INPUT);
      d.g->err_index = u;
      x = 0.0;
    }
    double f = x / bx.L[k];
    const double fl = floor(f);
    im[k] = (int)fl;
    f -= fl;
    if (f >= 1.0) f -= 1.0;
    if (f < 0.0) f = 0.0;
    p[k] = frac64_of(f);
  }
  d.x[i] = p[0];
  d.y[i] = p[1];
  d.z[i] = p[2];
  if (d.img) d.img[i] = make_int4(im[0], im[1], im[2], 0);
  const uint4 q = make_uint4(q_of(p[0]), q_of(p[1]), q_of(p[2]), (unsigned)b);
  d.q[i] = q;
  if (d.typ) d.typ[i] = d.utyp[u];
  d.f[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  const uint4 qb = d.qb[i];
  const float dx = fix_diff(qb.x, q.x, bx.Lq[0]), dy = fix_diff(qb.y, q.y, bx.Lq[1]), dz = fix_diff(qb.z, q.z, bx.Lq[2]);
  if (fmaf(dx, dx, fmaf(dy, dy, dz * dz)) > hs2) {
    d.bst[b].rebuild = 1;
    d.g->any_rebuild = 1;
  }
}

__device__ __forceinline__ float load_keep_velocity(const Dev& d, const Integ& I, const double* __restrict__ vin,
                                                    int i) {
  const int u = d.id[i];
  float vh[3];
  for (int k = 0; k < 3; ++k) {
    double w = vin ? vin[3 * (size_t)u + k] : 0.0;
    if (!isfinite(w)) {
      set_status(d.g, ST_INPUT);
      d.g->err_index = u;
      w = 0.0;
    }
    const float2 sw = split_df(w);
    (k == 0 ? d.vx : (k == 1 ? d.vy : d.vz))[i] = sw;
    vh[k] = sw.x + sw.y;
  }
  return (float)I.ke_fac * fmaf(vh[0], vh[0], fmaf(vh[1], vh[1], vh[2] * vh[2]));
}

__global__ void k_load_state_keep(Dev d, const double* __restrict__ xin, const double* __restrict__ vin,
                                  int count_terms, float hs2) {
  const Integ I = *d.integ;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < d.ncell) d.cell_cnt[i] = 0;
  if (i < d.nbox) {
    d.bst[i].s_endc = 1.0;
    d.bst[i].Lb = d.box[i].L[0];  // the lists were built in these (unscaled) boxes
  }
  if (i == 0) d.g->count_terms = count_terms;
  float ke[1] = {0.f};
  int b = -1;
  if (i < d.N) {
    b = (int)d.q[i].w;
    load_keep_position(d, xin, i, hs2);
    ke[0] = load_keep_velocity(d, I, vin, i);
  }
  box_accumulate<1>(ke, b, [&](int bb) { return &d.bst[bb].ke_last; });
}

// The same in two launches, positions first (k_load_positions_keep: no
// velocity or kinetic energy is touched) and velocities later
// (k_load_velocities_keep: the kinetic energy into ke_last, which the host
// zeroed with the box states), so that a force call at the new positions can
// run between them while the velocities are still being copied in.
__global__ void k_load_positions_keep(Dev d, const double* __restrict__ xin, int count_terms, float hs2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < d.ncell) d.cell_cnt[i] = 0;
  if (i < d.nbox) {
    d.bst[i].s_endc = 1.0;
    d.bst[i].Lb = d.box[i].L[0];
  }
  if (i == 0) d.g->count_terms = count_terms;
  if (i < d.N) load_keep_position(d, xin, i, hs2);
}

__global__ void k_load_velocities_keep(Dev d, const double* __restrict__ vin) {
  const Integ I = *d.integ;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  float ke[1] = {0.f};
  int b = -1;
  if (i < d.N) {
    b = (int)d.q[i].w;
    ke[0] = load_keep_velocity(d, I, vin, i);
  }
  box_accumulate<1>(ke, b, [&](int bb) { return &d.bst[bb].ke_last; });
}

// Applies a pending second half-kick (v += dt/2 F/m) before anything changes
// the forces or the atom order outside a step.
__global__ void k_flush_pending(Dev d) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (!d.g->pend) return;
  const double cf = d.integ->cf;
  if (i < d.N) {
    const float4 F = d.f[i];
    d.vx[i] = split_df(join_df(d.vx[i]) + cf * F.x);
    d.vy[i] = split_df(join_df(d.vy[i]) + cf * F.y);
    d.vz[i] = split_df(join_df(d.vz[i]) + cf * F.z);
  }
}

// Flags every box for a rebuild (new state, parameters, skin or list width).
__global__ void k_flag_all(Dev d) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < d.nbox) d.bst[b].rebuild = 1;
  if (b == 0) d.g->any_rebuild = 1;
}

// Blocks of the standalone kick kernels: `items` atoms per thread.
__host__ __device__ inline int kick_blocks(int n, int threads, int items = 1) {
  const int per = threads * items;
  return (n + per - 1) / per;
}

// Zeroes this parity's energy/virial accumulators and (optionally) the forces.
__global__ void k_prep_force(Dev d, int zero_f) {
  const int par = (int)(d.g->step & 1ull);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) {
    d.g->n_over = 0;
    d.g->npairs = 0;
    d.g->ntrip = 0;
  }
  if (i < d.nbox)
    for (int k = 0; k < 8; ++k) d.bst[i].ew[par][k] = 0.0;
  if (zero_f && i < d.N) d.f[i] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// Thermo record from the current accumulators without advancing (forces just
// evaluated).
__global__ void k_thermo_snapshot(Dev d) {
  const Integ I = *d.integ;
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= d.nbox) return;
  const int par = (int)(d.g->step & 1ull);
  const BoxState* st = d.bst + b;
  const Box& bx = d.box[b];
  double* t = d.thermo + (size_t)b * TR_N;
  const double ke = st->ke_last;
  const double e2 = st->ew[par][0], e3 = st->ew[par][1];
  t[TR_STEP] = (double)d.g->step;
  t[TR_PE] = e2 + e3;
  t[TR_E2] = e2;
  t[TR_E3] = e3;
  t[TR_KE] = ke;
  t[TR_T] = 2.0 * ke * bx.inv_ndf_kb;
  double cons = ke + e2 + e3;
  const double xi = (double)st->th_e.x + (double)st->th_e.y, eta = (double)st->th_e.z + (double)st->th_e.w;
  if (I.kind == TH_NH || I.kind == TH_NPT) cons += 0.5 * bx.Q * xi * xi + bx.ndfkT0 * eta;
  if (I.kind == TH_NPT) cons += I.p_ext * bx.volume + 0.5 * st->pe_e * st->pe_e / bx.W;
  t[TR_CONS] = cons;
  t[TR_P] = (2.0 * ke + st->ew[par][2] + st->ew[par][3] + st->ew[par][4]) / (3.0 * bx.volume) * kATM;
  for (int k = 0; k < 6; ++k) t[TR_W0 + k] = st->ew[par][2 + k];
  t[TR_XI] = xi;
  t[TR_ETA] = eta;
  t[TR_REBUILDS] = (double)st->rebuilds;
  t[TR_VOL] = bx.volume;
  for (int k = 0; k < 3; ++k) t[TR_L0 + k] = bx.L[k];
}

// Sorted -> user order: x (wrapped) and (v + pending half-kick) * s_endc (the
// end scale of the last step, pending on the stored velocities).
__global__ void k_gather_state(Dev d, double* __restrict__ xo, double* __restrict__ vo, int unwrap) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.N) return;
  const int u = d.id[i];
  const Box& bx = d.box[d.q[i].w];
  if (xo) {
    constexpr double k2m64 = 5.421010862427522170037264e-20;  // 2^-64
    const int4 im = unwrap ? d.img[i] : make_int4(0, 0, 0, 0);
    xo[3 * (size_t)u] = (__ull2double_rn(d.x[i]) * k2m64 + im.x) * bx.L[0];
    xo[3 * (size_t)u + 1] = (__ull2double_rn(d.y[i]) * k2m64 + im.y) * bx.L[1];
    xo[3 * (size_t)u + 2] = (__ull2double_rn(d.z[i]) * k2m64 + im.z) * bx.L[2];
  }
  if (vo) {  // pending half-kick and end-of-step thermostat scale applied
    const double s = d.bst[d.q[i].w].s_endc;
    const double cf = d.g->pend ? d.integ->cf : 0.0;
    const float4 F = d.f[i];
    vo[3 * (size_t)u] = (join_df(d.vx[i]) + cf * F.x) * s;
    vo[3 * (size_t)u + 1] = (join_df(d.vy[i]) + cf * F.y) * s;
    vo[3 * (size_t)u + 2] = (join_df(d.vz[i]) + cf * F.z) * s;
  }
}

__global__ void k_gather_forces(Dev d, double* __restrict__ fo64, float* __restrict__ fo32) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.N) return;
  const int u = d.id[i];
  const float4 F = d.f[i];
  if (fo64) {
    fo64[3 * (size_t)u] = F.x;
    fo64[3 * (size_t)u + 1] = F.y;
    fo64[3 * (size_t)u + 2] = F.z;
  }
  if (fo32) {
    fo32[3 * (size_t)u] = F.x;
    fo32[3 * (size_t)u + 1] = F.y;
    fo32[3 * (size_t)u + 2] = F.z;
  }
}

// Neighbour sets to user order: out[u*width + s] = id[nbr[i][s]].
__global__ void k_gather_neighbors(Dev d, int* __restrict__ cnt_out, int* __restrict__ nbr_out, int width) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.N) return;
  const int u = d.id[i];
  const int c = d.nbr_cnt[i];
  cnt_out[u] = c;
  const int m = min(min(c, d.W), width);
  for (int s = 0; s < m; ++s) nbr_out[(size_t)u * width + s] = d.id[d.nbr[(size_t)i * d.W + s]];
}

// Energies and virial of the latest force evaluation: the parity slot that
// evaluation wrote (wpar).  After a step the step counter has moved on and
// its own parity names the slot the next step clears, not this one.
__global__ void k_energy_out(Dev d, double* e, double* w) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= d.nbox) return;
  const int par = d.g->wpar;
  const BoxState* st = d.bst + b;
  if (e) {
    e[3 * b] = st->ew[par][0] + st->ew[par][1];
    e[3 * b + 1] = st->ew[par][0];
    e[3 * b + 2] = st->ew[par][1];
  }
  if (w)
    for (int k = 0; k < 6; ++k) w[6 * b + k] = st->ew[par][2 + k];
}

}  // namespace mw
