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
//   x,y,z,vx,vy,vz   FP64 master positions / velocities (SoA)
//   q                uint4 {qx, qy, qz, box}: position as a 32-bit fraction of
//                    the box edge; the minimum-image difference of two atoms
//                    is the wrapping int32 difference, converted once to FP32
//   f                float4 forces (w unused), accumulated with red.global
//   nbr              int32 [W][N] neighbour list (slot-major), nbr_cnt[N]
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
enum : int { ST_OK = 0, ST_OVERFLOW = 3, ST_NAN = 4, ST_LOST = 5, ST_TIMEOUT = 6, ST_LEGS = 10 };

enum : int { TH_NVE = 0, TH_BERENDSEN = 1, TH_NH = 2 };

// Legs kept in registers per centre atom in the fused force kernel; centres
// with more legs take the overflow path.
constexpr int kMaxLegs = 16;
// Upper bound for the overflow path (more legs than this = overlapping atoms).
constexpr int kMaxLegsOverflow = 64;

struct Box {        // read-only in kernels
  double L[3];
  double qs[3];     // 2^32 / L
  float Lq[3];      // L / 2^32
  int off, n;       // atom range
  int nc[3];        // cells per dimension
  int cell_off;     // first global cell
  double T0, Ndf, Q, volume;
};

struct BoxState {   // mutated by kernels
  double xi[2], eta[2];   // [0] after the end-of-step half, [1] after the start-of-step half
  double s_end;           // pending velocity scale: true v = stored v * s_end
  double ke_last;         // kinetic energy after the last end half (kcal/mol)
  double ke_acc[2];       // per step-parity accumulators of the raw kinetic energy
  double ew[2][8];        // per step-parity E2, E3, W[6]
  int rebuild;            // displacement flag of this box
  int pad_;
  long long rebuilds;
};

// Per-box thermo record written at the end of each step (doubles).
enum { TR_STEP, TR_PE, TR_E2, TR_E3, TR_KE, TR_T, TR_CONS, TR_P, TR_W0, TR_XI = TR_W0 + 6, TR_ETA,
       TR_REBUILDS, TR_N };

struct Global {
  unsigned long long step;  // completed steps since set_state
  int any_rebuild;
  int status;
  int max_count;            // widest neighbour set of the last build
  unsigned done;            // last-block counter of k_kick2
  unsigned bar_count, bar_gen;
  long long npairs, ntrip;  // leg / triplet counts of the last force call (if counting)
  int count_terms;
  int n_over;               // centres routed to the overflow path
  int err_index;
  int pad_;
};

struct Integ {
  double dt;
  double cf;         // 0.5 dt FCONV / mass
  double ke_fac;     // 0.5 mass / FCONV
  double tau;
  int kind;
  float half_skin2;  // (skin/2)^2
};

struct FParams {     // FP32 constants of the force kernels
  float rc, rc2, rl2;
  float sig, sig_l2e, gsig_l2e, gsig;
  float Aeps, B, c0, sle;  // sle = sqrt(lambda eps)
  int p, q;
};

struct Dev {
  int N, W, ncell, nbox;
  double *x, *y, *z, *vx, *vy, *vz;
  double *tx, *ty, *tz, *tvx, *tvy, *tvz;
  uint4 *q, *qb, *tq;
  float4* f;
  int *id, *tid;
  int *cell, *rank;
  int *cell_cnt, *cell_start;
  int *nbr, *nbr_cnt;
  int* over;          // overflow centre list
  const Box* box;
  BoxState* bst;
  double* thermo;     // nbox * TR_N
  Global* g;
  const Integ* integ;
  double* stage;      // n*3 doubles staging (user order)
  double* stage2;
};

// ---------------------------------------------------------------------------
// small helpers

__device__ __forceinline__ uint32_t to_fixed(double x, double qs) {
  return (uint32_t)(unsigned long long)__double2ll_rn(x * qs);
}

__device__ __forceinline__ float fix_diff(uint32_t a, uint32_t b, float lq) {  // b - a, minimum image
  return __int2float_rn((int)(b - a)) * lq;
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

__device__ __forceinline__ int cell_of(const uint4& q, const Box& bx) {
  const int cx = (int)(((unsigned long long)q.x * (unsigned)bx.nc[0]) >> 32);
  const int cy = (int)(((unsigned long long)q.y * (unsigned)bx.nc[1]) >> 32);
  const int cz = (int)(((unsigned long long)q.z * (unsigned)bx.nc[2]) >> 32);
  return bx.cell_off + cx + bx.nc[0] * (cy + bx.nc[1] * cz);
}

__device__ __forceinline__ void set_status(Global* g, int st) { atomicCAS(&g->status, 0, st); }

// Per-box FP64 accumulation of NV values.  Every thread of the block calls it
// (b < 0 for threads without an atom).  Atoms are box-major, so the box ids
// along a warp are non-decreasing: a segmented warp scan sums each box run;
// runs of the block's first and last box are merged in shared memory and
// flushed with one global atomic per value, other runs go to global directly.
template <int NV, class Dst>
__device__ void box_accumulate(double (&v)[NV], int b, bool is_last_valid, Dst dst) {
  __shared__ double sacc[2][NV];
  __shared__ int sbox[2];
  const int lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    sbox[0] = b;
    sbox[1] = -1;
  }
  if (threadIdx.x < 2 * NV) (&sacc[0][0])[threadIdx.x] = 0.0;
  __syncthreads();
  if (is_last_valid) sbox[1] = b;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const int bo = __shfl_up_sync(kFull, b, off);
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      const double vo = __shfl_up_sync(kFull, v[k], off);
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
      for (int k = 0; k < NV; ++k) atomicAdd(p + k, v[k]);
    }
  }
  __syncthreads();
  if (threadIdx.x < NV && sbox[0] >= 0) atomicAdd(dst(sbox[0]) + threadIdx.x, sacc[0][threadIdx.x]);
  if (threadIdx.x >= 32 && threadIdx.x < 32 + NV && sbox[1] >= 0 && sbox[1] != sbox[0])
    atomicAdd(dst(sbox[1]) + (threadIdx.x - 32), sacc[1][threadIdx.x - 32]);
}

// One Nose-Hoover half step (length dt/2) of a single thermostat: quarter step
// on xi, velocity scale exp(-xi dt/2), half step on eta, quarter step on xi.
__device__ __forceinline__ double nh_half(double& ke, double& xi, double& eta, double dt, double Ndf, double kT0,
                                          double Q) {
  xi += 0.25 * dt * (2.0 * ke - Ndf * kT0) / Q;
  const double s = exp(-xi * 0.5 * dt);
  ke *= s * s;
  eta += xi * 0.5 * dt;
  xi += 0.25 * dt * (2.0 * ke - Ndf * kT0) / Q;
  return s;
}

// Velocity scale applied at the start of a step for box b: the pending
// end-of-step scale of the previous step times this step's start-half scale.
// The writer (the thread owning the box's first atom) also stores the
// thermostat state after the start half and clears this step's accumulators.
__device__ double kick1_scale_of_box(const Dev& d, int b, const Integ& I, bool writer, int par) {
  BoxState* st = d.bst + b;
  const Box& bx = d.box[b];
  double s = st->s_end;
  double xi = st->xi[0], eta = st->eta[0];
  if (I.kind == TH_NH) {
    double ke = st->ke_last;
    s *= nh_half(ke, xi, eta, I.dt, bx.Ndf, kKB * bx.T0, bx.Q);
  }
  if (writer) {
    st->xi[1] = xi;
    st->eta[1] = eta;
    st->ke_acc[par] = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) st->ew[par][k] = 0.0;
  }
  return s;
}

// ---------------------------------------------------------------------------
// Phase bodies (one item each) shared by the per-phase kernels and the
// persistent kernel.

// a1 + a7 (first half): v = v*s + dt/2 a; x += dt v; wrap; fixed-point copy;
// displacement check against the last build.  Also zeroes f for this step.
__device__ __forceinline__ void kick1_item(const Dev& d, const Integ& I, int i, double s, int b) {
  const Box& bx = d.box[b];
  const float4 F = d.f[i];
  d.f[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  const double vx = d.vx[i] * s + I.cf * (double)F.x;
  const double vy = d.vy[i] * s + I.cf * (double)F.y;
  const double vz = d.vz[i] * s + I.cf * (double)F.z;
  double px = d.x[i] + I.dt * vx, py = d.y[i] + I.dt * vy, pz = d.z[i] + I.dt * vz;
  if (px >= bx.L[0]) px -= bx.L[0]; else if (px < 0.0) px += bx.L[0];
  if (py >= bx.L[1]) py -= bx.L[1]; else if (py < 0.0) py += bx.L[1];
  if (pz >= bx.L[2]) pz -= bx.L[2]; else if (pz < 0.0) pz += bx.L[2];
  d.vx[i] = vx; d.vy[i] = vy; d.vz[i] = vz;
  d.x[i] = px; d.y[i] = py; d.z[i] = pz;
  const uint4 qn = make_uint4(to_fixed(px, bx.qs[0]), to_fixed(py, bx.qs[1]), to_fixed(pz, bx.qs[2]), (unsigned)b);
  d.q[i] = qn;
  const uint4 qb = d.qb[i];
  const float dx = fix_diff(qb.x, qn.x, bx.Lq[0]);
  const float dy = fix_diff(qb.y, qn.y, bx.Lq[1]);
  const float dz = fix_diff(qb.z, qn.z, bx.Lq[2]);
  if (fmaf(dx, dx, fmaf(dy, dy, dz * dz)) > I.half_skin2) {
    d.bst[b].rebuild = 1;
    d.g->any_rebuild = 1;
  }
  const double step2 = I.dt * I.dt * (vx * vx + vy * vy + vz * vz);
  const double lmin = fmin(bx.L[0], fmin(bx.L[1], bx.L[2]));
  if (!(step2 < 0.25 * lmin * lmin)) {
    set_status(d.g, (step2 == step2) ? ST_LOST : ST_NAN);
    d.g->err_index = i;
  }
}

// Warp-cooperative scale: one evaluation per distinct box in the warp.
__device__ __forceinline__ double warp_kick1_scale(const Dev& d, const Integ& I, int i, int b, int par) {
  const int lane = threadIdx.x & 31;
  const int b0 = __shfl_sync(kFull, b, 0);
  const bool uni = __all_sync(kFull, b == b0 || b < 0);
  if (uni) {
    double t = 1.0;
    if (lane == 0 && b0 >= 0) t = kick1_scale_of_box(d, b0, I, i == d.box[b0].off, par);
    return __shfl_sync(kFull, t, 0);
  }
  return (b >= 0) ? kick1_scale_of_box(d, b, I, i == d.box[b].off, par) : 1.0;
}

// a7 (second half) for one atom; returns its raw kinetic energy.
__device__ __forceinline__ double kick2_item(const Dev& d, const Integ& I, int i) {
  const float4 F = d.f[i];
  const double vx = d.vx[i] + I.cf * (double)F.x;
  const double vy = d.vy[i] + I.cf * (double)F.y;
  const double vz = d.vz[i] + I.cf * (double)F.z;
  d.vx[i] = vx; d.vy[i] = vy; d.vz[i] = vz;
  const double ke = I.ke_fac * (vx * vx + vy * vy + vz * vz);
  if (!(ke < 1e30)) {
    set_status(d.g, ST_NAN);
    d.g->err_index = i;
  }
  return ke;
}

// End-of-step thermostat half and thermo record of box b (one thread per box).
__device__ void end_of_step_box(const Dev& d, const Integ& I, int b, int par, unsigned long long step_done) {
  BoxState* st = d.bst + b;
  const Box& bx = d.box[b];
  double ke = __ldcg(&st->ke_acc[par]);
  double xi = st->xi[1], eta = st->eta[1];
  double s = 1.0;
  if (I.kind == TH_NH) {
    s = nh_half(ke, xi, eta, I.dt, bx.Ndf, kKB * bx.T0, bx.Q);
  } else if (I.kind == TH_BERENDSEN) {
    const double T = 2.0 * ke / (bx.Ndf * kKB);
    if (T > 0.0) {
      s = sqrt(1.0 + I.dt / I.tau * (bx.T0 / T - 1.0));
      ke *= s * s;
    }
  }
  st->s_end = s;
  st->ke_last = ke;
  st->xi[0] = xi;
  st->eta[0] = eta;
  double* t = d.thermo + (size_t)b * TR_N;
  const double e2 = __ldcg(&st->ew[par][0]), e3 = __ldcg(&st->ew[par][1]);
  double w[6];
  for (int k = 0; k < 6; ++k) w[k] = __ldcg(&st->ew[par][2 + k]);
  t[TR_STEP] = (double)step_done;
  t[TR_PE] = e2 + e3;
  t[TR_E2] = e2;
  t[TR_E3] = e3;
  t[TR_KE] = ke;
  t[TR_T] = 2.0 * ke / (bx.Ndf * kKB);
  double cons = ke + e2 + e3;
  if (I.kind == TH_NH) cons += 0.5 * bx.Q * xi * xi + bx.Ndf * kKB * bx.T0 * eta;
  t[TR_CONS] = cons;
  t[TR_P] = (2.0 * ke + w[0] + w[1] + w[2]) / (3.0 * bx.volume) * kATM;
  for (int k = 0; k < 6; ++k) t[TR_W0 + k] = w[k];
  t[TR_XI] = xi;
  t[TR_ETA] = eta;
  t[TR_REBUILDS] = (double)st->rebuilds;
}

// ---------------------------------------------------------------------------
// Neighbour list: one warp per centre atom, candidates of the (deduplicated)
// 27-cell stencil flattened over the lanes, ballot + popc compaction.
__device__ __forceinline__ int stencil_n(int nc) { return nc >= 3 ? 3 : nc; }
__device__ __forceinline__ int stencil_off(int nc, int o) { return nc >= 3 ? o - 1 : o; }

__device__ void neigh_warp(const Dev& d, int i, float rl2) {
  const int lane = threadIdx.x & 31;
  const uint4 qi = d.q[i];
  const Box& bx = d.box[qi.w];
  const int cx = (int)(((unsigned long long)qi.x * (unsigned)bx.nc[0]) >> 32);
  const int cy = (int)(((unsigned long long)qi.y * (unsigned)bx.nc[1]) >> 32);
  const int cz = (int)(((unsigned long long)qi.z * (unsigned)bx.nc[2]) >> 32);
  const int nx = stencil_n(bx.nc[0]), ny = stencil_n(bx.nc[1]), nz = stencil_n(bx.nc[2]);
  int start = 0, cnt = 0;
  if (lane < nx * ny * nz) {
    const int ox = lane % nx, oy = (lane / nx) % ny, oz = lane / (nx * ny);
    const int X = (cx + stencil_off(bx.nc[0], ox) + bx.nc[0]) % bx.nc[0];
    const int Y = (cy + stencil_off(bx.nc[1], oy) + bx.nc[1]) % bx.nc[1];
    const int Z = (cz + stencil_off(bx.nc[2], oz) + bx.nc[2]) % bx.nc[2];
    const int c = bx.cell_off + X + bx.nc[0] * (Y + bx.nc[1] * Z);
    start = d.cell_start[c];
    cnt = d.cell_start[c + 1] - start;
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
  int m = 0;
  for (int base = 0; base < total; base += 32) {
    const int t = base + lane;
    int lo = 0, hi = 31;
#pragma unroll
    for (int it = 0; it < 5; ++it) {  // smallest lane k with incl_k > t
      const int mid = (lo + hi) >> 1;
      const int v = __shfl_sync(kFull, incl, mid);
      if (v > t) hi = mid; else lo = mid + 1;
    }
    const int sk = __shfl_sync(kFull, start, lo);
    const int ek = __shfl_sync(kFull, excl, lo);
    bool pred = false;
    int j = 0;
    if (t < total) {
      j = sk + (t - ek);
      if (j != i) {
        const uint4 qj = d.q[j];
        const float dx = fix_diff(qi.x, qj.x, L0), dy = fix_diff(qi.y, qj.y, L1), dz = fix_diff(qi.z, qj.z, L2);
        pred = fmaf(dx, dx, fmaf(dy, dy, dz * dz)) < rl2;
      }
    }
    const unsigned bal = __ballot_sync(kFull, pred);
    const int pos = m + __popc(bal & ((1u << lane) - 1u));
    if (pred && pos < d.W) d.nbr[(size_t)pos * d.N + i] = j;
    m += __popc(bal);
  }
  if (lane == 0) {
    d.nbr_cnt[i] = m;
    atomicMax(&d.g->max_count, m);
    if (m > d.W) set_status(d.g, ST_OVERFLOW);
  }
}

// ---------------------------------------------------------------------------
// Fused two- + three-body force.  One thread per centre atom i:
//   pass 1: walk the neighbour list, keep legs r < a sig; pair term (owner
//           computes: half energy, full force on i, half virial); stage leg
//           data in shared memory;
//   pass 2: legs to registers (compile-time indices);
//   pass 3: all leg pairs j < k: three-body energy and forces on j and k;
//   pass 4: scatter leg forces with red.global.add.v4.f32, force on i,
//           per-leg virial; FP64 per-box reduction of E2, E3, W.
// Leg data: u (unit vector i->j), tr = 2/r, nde = gam sig/(r - a sig)^2,
// ee = sqrt(lam eps) exp(gam sig/(r - a sig)).
//   phi3 = ee_j ee_k D^2, D = u_j.u_k - cos th0
//   F_j  = -g [tr_j (u_k - c u_j) - D nde_j u_j],  g = ee_j ee_k D
constexpr int kForceThreads = 128;

struct LegSm {  // shared-memory leg staging, field-major per thread for conflict-free access
  float v[8][kMaxLegs][kForceThreads];
};

template <bool kCount>
__device__ __forceinline__ void force_item(const Dev& d, const FParams& P, int i, LegSm* sm, float (&acc)[8],
                                           int& nl_out) {
  const int t = threadIdx.x;
  const uint4 qi = d.q[i];
  const Box& bx = d.box[qi.w];
  const float L0 = bx.Lq[0], L1 = bx.Lq[1], L2 = bx.Lq[2];
  int cnt = d.nbr_cnt[i];
  if (cnt > d.W) cnt = d.W;
  float fix = 0.f, fiy = 0.f, fiz = 0.f;
  int nl = 0;
  for (int s = 0; s < cnt; ++s) {
    const int j = __ldg(d.nbr + (size_t)s * d.N + i);
    const uint4 qj = d.q[j];
    const float dx = fix_diff(qi.x, qj.x, L0), dy = fix_diff(qi.y, qj.y, L1), dz = fix_diff(qi.z, qj.z, L2);
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    if (r2 >= P.rc2) continue;
    const float invr = rsqrtf(r2);
    const float r = r2 * invr;
    if (!(r < P.rc)) continue;
    const float ux = dx * invr, uy = dy * invr, uz = dz * invr;
    const float tinv = __frcp_rn(r - P.rc);  // 1/(r - a sig) < 0
    const float e2 = exp2f(P.sig_l2e * tinv);
    const float e3 = exp2f(P.gsig_l2e * tinv);
    const float sr = P.sig * invr;
    const float srp = powi(sr, P.p), srq = powi(sr, P.q);
    const float brk = fmaf(P.B, srp, -srq);
    const float phi = P.Aeps * brk * e2;
    const float dphi = P.Aeps * e2 * fmaf((float)(-P.p) * P.B, srp, (float)P.q * srq) * invr -
                       P.Aeps * e2 * brk * P.sig * tinv * tinv;
    acc[0] = fmaf(0.5f, phi, acc[0]);
    fix = fmaf(dphi, ux, fix);
    fiy = fmaf(dphi, uy, fiy);
    fiz = fmaf(dphi, uz, fiz);
    const float wv = -0.5f * dphi * r;
    acc[2] = fmaf(wv * ux, ux, acc[2]);
    acc[3] = fmaf(wv * uy, uy, acc[3]);
    acc[4] = fmaf(wv * uz, uz, acc[4]);
    acc[5] = fmaf(wv * ux, uy, acc[5]);
    acc[6] = fmaf(wv * ux, uz, acc[6]);
    acc[7] = fmaf(wv * uy, uz, acc[7]);
    if (nl < kMaxLegs) {
      sm->v[0][nl][t] = ux;
      sm->v[1][nl][t] = uy;
      sm->v[2][nl][t] = uz;
      sm->v[3][nl][t] = 2.0f * invr;
      sm->v[4][nl][t] = P.gsig * tinv * tinv;
      sm->v[5][nl][t] = P.sle * e3;
      sm->v[6][nl][t] = r;
      sm->v[7][nl][t] = __int_as_float(j);
    }
    ++nl;
  }
  nl_out = nl;
  if (kCount) {
    atomicAdd((unsigned long long*)&d.g->npairs, (unsigned long long)nl);
  }
  if (nl > kMaxLegs) {
    // three-body part handled by the overflow kernel; pair part is complete
    red_add_v4(d.f + i, fix, fiy, fiz);
    const int slot = atomicAdd(&d.g->n_over, 1);
    if (slot < d.N) d.over[slot] = i;
    return;
  }
  if (kCount) atomicAdd((unsigned long long*)&d.g->ntrip, (unsigned long long)(nl * (nl - 1) / 2));
  float ux[kMaxLegs], uy[kMaxLegs], uz[kMaxLegs], tr[kMaxLegs], nde[kMaxLegs], ee[kMaxLegs];
  float ax[kMaxLegs], ay[kMaxLegs], az[kMaxLegs];
#pragma unroll
  for (int k = 0; k < kMaxLegs; ++k) {
    ax[k] = ay[k] = az[k] = 0.f;
    if (k < nl) {
      ux[k] = sm->v[0][k][t];
      uy[k] = sm->v[1][k][t];
      uz[k] = sm->v[2][k][t];
      tr[k] = sm->v[3][k][t];
      nde[k] = sm->v[4][k][t];
      ee[k] = sm->v[5][k][t];
    } else {
      ux[k] = uy[k] = uz[k] = tr[k] = nde[k] = ee[k] = 0.f;
    }
  }
  float e3acc = 0.f;
  const float c0 = P.c0;
#pragma unroll
  for (int j = 0; j < kMaxLegs - 1; ++j) {
    if (j + 1 >= nl) break;
#pragma unroll
    for (int k = j + 1; k < kMaxLegs; ++k) {
      if (k >= nl) break;
      const float c = fmaf(ux[j], ux[k], fmaf(uy[j], uy[k], uz[j] * uz[k]));
      const float D = c - c0;
      const float g = ee[j] * ee[k] * D;
      e3acc = fmaf(g, D, e3acc);
      const float aj = g * tr[j];
      const float bj = g * fmaf(c, tr[j], D * nde[j]);  // = -(g (D de_j - c tr_j)), de = -nde
      ax[j] = fmaf(-aj, ux[k], fmaf(bj, ux[j], ax[j]));
      ay[j] = fmaf(-aj, uy[k], fmaf(bj, uy[j], ay[j]));
      az[j] = fmaf(-aj, uz[k], fmaf(bj, uz[j], az[j]));
      const float ak = g * tr[k];
      const float bk = g * fmaf(c, tr[k], D * nde[k]);
      ax[k] = fmaf(-ak, ux[j], fmaf(bk, ux[k], ax[k]));
      ay[k] = fmaf(-ak, uy[j], fmaf(bk, uy[k], ay[k]));
      az[k] = fmaf(-ak, uz[j], fmaf(bk, uz[k], az[k]));
    }
  }
  acc[1] += e3acc;
#pragma unroll
  for (int k = 0; k < kMaxLegs; ++k) {
    if (k >= nl) break;
    const int j = __float_as_int(sm->v[7][k][t]);
    const float r = sm->v[6][k][t];
    red_add_v4(d.f + j, ax[k], ay[k], az[k]);
    fix -= ax[k];
    fiy -= ay[k];
    fiz -= az[k];
    const float rx = r * ux[k], ry = r * uy[k], rz = r * uz[k];
    acc[2] = fmaf(rx, ax[k], acc[2]);
    acc[3] = fmaf(ry, ay[k], acc[3]);
    acc[4] = fmaf(rz, az[k], acc[4]);
    acc[5] = fmaf(rx, ay[k], acc[5]);
    acc[6] = fmaf(rx, az[k], acc[6]);
    acc[7] = fmaf(ry, az[k], acc[7]);
  }
  red_add_v4(d.f + i, fix, fiy, fiz);
}

// Three-body part for centres with more than kMaxLegs legs (rare): legs in
// local memory, same arithmetic.
template <bool kCount>
__device__ void force_overflow_item(const Dev& d, const FParams& P, int i, float (&acc)[8]) {
  const uint4 qi = d.q[i];
  const Box& bx = d.box[qi.w];
  int cnt = d.nbr_cnt[i];
  if (cnt > d.W) cnt = d.W;
  float ux[kMaxLegsOverflow], uy[kMaxLegsOverflow], uz[kMaxLegsOverflow], tr[kMaxLegsOverflow],
      nde[kMaxLegsOverflow], ee[kMaxLegsOverflow], rr[kMaxLegsOverflow];
  float ax[kMaxLegsOverflow], ay[kMaxLegsOverflow], az[kMaxLegsOverflow];
  int jj[kMaxLegsOverflow];
  int nl = 0;
  for (int s = 0; s < cnt; ++s) {
    const int j = d.nbr[(size_t)s * d.N + i];
    const uint4 qj = d.q[j];
    const float dx = fix_diff(qi.x, qj.x, bx.Lq[0]), dy = fix_diff(qi.y, qj.y, bx.Lq[1]),
                dz = fix_diff(qi.z, qj.z, bx.Lq[2]);
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    if (r2 >= P.rc2) continue;
    const float invr = rsqrtf(r2);
    const float r = r2 * invr;
    if (!(r < P.rc)) continue;
    if (nl >= kMaxLegsOverflow) {
      set_status(d.g, ST_LEGS);
      d.g->err_index = i;
      return;
    }
    const float tinv = __frcp_rn(r - P.rc);
    ux[nl] = dx * invr;
    uy[nl] = dy * invr;
    uz[nl] = dz * invr;
    tr[nl] = 2.0f * invr;
    nde[nl] = P.gsig * tinv * tinv;
    ee[nl] = P.sle * exp2f(P.gsig_l2e * tinv);
    rr[nl] = r;
    jj[nl] = j;
    ax[nl] = ay[nl] = az[nl] = 0.f;
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
  acc[1] += e3acc;
  float fx = 0.f, fy = 0.f, fz = 0.f;
  for (int k = 0; k < nl; ++k) {
    red_add_v4(d.f + jj[k], ax[k], ay[k], az[k]);
    fx -= ax[k];
    fy -= ay[k];
    fz -= az[k];
    const float rx = rr[k] * ux[k], ry = rr[k] * uy[k], rz = rr[k] * uz[k];
    acc[2] = fmaf(rx, ax[k], acc[2]);
    acc[3] = fmaf(ry, ay[k], acc[3]);
    acc[4] = fmaf(rz, az[k], acc[4]);
    acc[5] = fmaf(rx, ay[k], acc[5]);
    acc[6] = fmaf(rx, az[k], acc[6]);
    acc[7] = fmaf(ry, az[k], acc[7]);
  }
  red_add_v4(d.f + i, fx, fy, fz);
}

// ---------------------------------------------------------------------------
// Per-phase kernels (the graph engine and the standalone force call).

__global__ void k_kick1(Dev d) {
  if (d.g->status) return;
  const Integ I = *d.integ;
  const int par = (int)(d.g->step & 1ull);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) d.g->n_over = 0;
  const int b = (i < d.N) ? (int)d.q[i].w : -1;
  const double s = warp_kick1_scale(d, I, i, b, par);
  if (i < d.N) kick1_item(d, I, i, s, b);
}

__global__ void k_bin(Dev d) {
  if (!d.g->any_rebuild || d.g->status) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) d.g->max_count = 0;
  if (i >= d.N) return;
  const uint4 q = d.q[i];
  const int c = cell_of(q, d.box[q.w]);
  d.cell[i] = c;
  d.rank[i] = atomicAdd(d.cell_cnt + c, 1);
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
  if (i >= d.N) return;
  const int p = d.cell_start[d.cell[i]] + d.rank[i];
  d.tx[p] = d.x[i]; d.ty[p] = d.y[i]; d.tz[p] = d.z[i];
  d.tvx[p] = d.vx[i]; d.tvy[p] = d.vy[i]; d.tvz[p] = d.vz[i];
  d.tid[p] = d.id[i];
  d.tq[p] = d.q[i];
}

__global__ void k_copyback(Dev d) {
  if (!d.g->any_rebuild || d.g->status) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < d.nbox) d.bst[i].rebuilds += 1;
  if (i >= d.N) return;
  d.x[i] = d.tx[i]; d.y[i] = d.ty[i]; d.z[i] = d.tz[i];
  d.vx[i] = d.tvx[i]; d.vy[i] = d.tvy[i]; d.vz[i] = d.tvz[i];
  d.id[i] = d.tid[i];
  const uint4 q = d.tq[i];
  d.q[i] = q;
  d.qb[i] = q;
}

__global__ void k_neigh(Dev d, float rl2) {
  if (!d.g->any_rebuild || d.g->status) return;
  const int w = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
  if (w >= d.N) return;
  neigh_warp(d, w, rl2);
}

template <bool kCount>
__global__ void __launch_bounds__(kForceThreads, 3) k_force(Dev d, FParams P) {
  if (d.g->status) return;
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  LegSm* sm = reinterpret_cast<LegSm*>(dyn_smem);
  const int par = (int)(d.g->step & 1ull);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  int b = -1, nl = 0;
  if (i < d.N) {
    b = (int)d.q[i].w;
    force_item<kCount>(d, P, i, sm, acc, nl);
  }
  if (blockIdx.x == 0) {  // the rebuild (if any) is consumed
    for (int k = threadIdx.x; k < d.nbox; k += blockDim.x) d.bst[k].rebuild = 0;
    if (threadIdx.x == 0) d.g->any_rebuild = 0;
  }
  double v[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) v[k] = (double)acc[k];
  const bool last = (i < d.N) && (threadIdx.x == blockDim.x - 1 || i == d.N - 1);
  box_accumulate<8>(v, b, last, [&](int bb) { return &d.bst[bb].ew[par][0]; });
}

template <bool kCount>
__global__ void __launch_bounds__(128) k_force_overflow(Dev d, FParams P) {
  if (d.g->status) return;
  const int par = (int)(d.g->step & 1ull);
  const int nover = min(d.g->n_over, d.N);
  for (int base = blockIdx.x * blockDim.x; base < nover; base += gridDim.x * blockDim.x) {
    const int k = base + threadIdx.x;
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    int b = -1;
    if (k < nover) {
      const int i = d.over[k];
      b = (int)d.q[i].w;
      force_overflow_item<kCount>(d, P, i, acc);
    }
    // overflow centres are not box-ordered: plain per-thread FP64 atomics
    if (b >= 0)
      for (int c = 0; c < 8; ++c) atomicAdd(&d.bst[b].ew[par][c], (double)acc[c]);
  }
  __syncthreads();
}

__global__ void k_kick2(Dev d) {
  if (d.g->status) return;
  const Integ I = *d.integ;
  const unsigned long long step = d.g->step;
  const int par = (int)(step & 1ull);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double ke[1] = {0.0};
  int b = -1;
  if (i < d.N) {
    b = (int)d.q[i].w;
    ke[0] = kick2_item(d, I, i);
  }
  const bool last = (i < d.N) && (threadIdx.x == blockDim.x - 1 || i == d.N - 1);
  box_accumulate<1>(ke, b, last, [&](int bb) { return &d.bst[bb].ke_acc[par]; });
  // last block finishes the step: end-of-step thermostat half per box
  __shared__ bool am_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) am_last = (atomicAdd(&d.g->done, 1u) == gridDim.x - 1);
  __syncthreads();
  if (am_last) {
    __threadfence();
    for (int bb = threadIdx.x; bb < d.nbox; bb += blockDim.x) end_of_step_box(d, I, bb, par, step + 1);
    __syncthreads();
    if (threadIdx.x == 0) {
      d.g->done = 0;
      d.g->step = step + 1;
    }
  }
}

// ---------------------------------------------------------------------------
// Setup / IO kernels.

// Positions from a user-order AoS array (host copy or device pointer) into the
// sorted arrays: x[i] = xin[id[i]], wrapped into [0, L); q recomputed.
__global__ void k_load_positions(Dev d, const double* __restrict__ xin, const int* __restrict__ boxid,
                                 int identity) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.N) return;
  if (identity) d.id[i] = i;
  const int u = d.id[i];
  const int b = boxid[u];
  const Box& bx = d.box[b];
  double p[3];
  for (int k = 0; k < 3; ++k) {
    double v = xin[3 * (size_t)u + k];
    v -= bx.L[k] * floor(v / bx.L[k]);
    if (v >= bx.L[k]) v -= bx.L[k];
    if (v < 0.0) v = 0.0;
    p[k] = v;
  }
  d.x[i] = p[0]; d.y[i] = p[1]; d.z[i] = p[2];
  d.q[i] = make_uint4(to_fixed(p[0], bx.qs[0]), to_fixed(p[1], bx.qs[1]), to_fixed(p[2], bx.qs[2]), (unsigned)b);
}

__global__ void k_load_velocities(Dev d, const double* __restrict__ vin) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.N) return;
  const int u = d.id[i];
  if (vin) {
    d.vx[i] = vin[3 * (size_t)u];
    d.vy[i] = vin[3 * (size_t)u + 1];
    d.vz[i] = vin[3 * (size_t)u + 2];
  } else {
    d.vx[i] = d.vy[i] = d.vz[i] = 0.0;
  }
}

// Kinetic energy per box straight into ke_last (zeroed by the host).
__global__ void k_ke_init(Dev d) {
  const Integ I = *d.integ;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double ke[1] = {0.0};
  int b = -1;
  if (i < d.N) {
    b = (int)d.q[i].w;
    ke[0] = I.ke_fac * (d.vx[i] * d.vx[i] + d.vy[i] * d.vy[i] + d.vz[i] * d.vz[i]);
  }
  const bool last = (i < d.N) && (threadIdx.x == blockDim.x - 1 || i == d.N - 1);
  box_accumulate<1>(ke, b, last, [&](int bb) { return &d.bst[bb].ke_last; });
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

// Thermo record from the current accumulators without advancing (state just set).
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
  t[TR_T] = 2.0 * ke / (bx.Ndf * kKB);
  double cons = ke + e2 + e3;
  if (I.kind == TH_NH) cons += 0.5 * bx.Q * st->xi[0] * st->xi[0] + bx.Ndf * kKB * bx.T0 * st->eta[0];
  t[TR_CONS] = cons;
  t[TR_P] = (2.0 * ke + st->ew[par][2] + st->ew[par][3] + st->ew[par][4]) / (3.0 * bx.volume) * kATM;
  for (int k = 0; k < 6; ++k) t[TR_W0 + k] = st->ew[par][2 + k];
  t[TR_XI] = st->xi[0];
  t[TR_ETA] = st->eta[0];
  t[TR_REBUILDS] = (double)st->rebuilds;
}

// Sorted -> user order: x (wrapped) and v * s_end (pending thermostat scale).
__global__ void k_gather_state(Dev d, double* __restrict__ xo, double* __restrict__ vo) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.N) return;
  const int u = d.id[i];
  if (xo) {
    xo[3 * (size_t)u] = d.x[i];
    xo[3 * (size_t)u + 1] = d.y[i];
    xo[3 * (size_t)u + 2] = d.z[i];
  }
  if (vo) {
    const double s = d.bst[d.q[i].w].s_end;
    vo[3 * (size_t)u] = d.vx[i] * s;
    vo[3 * (size_t)u + 1] = d.vy[i] * s;
    vo[3 * (size_t)u + 2] = d.vz[i] * s;
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

// Neighbour sets to user order: out[u*width + s] = id[nbr[s][i]].
__global__ void k_gather_neighbors(Dev d, int* __restrict__ cnt_out, int* __restrict__ nbr_out, int width) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.N) return;
  const int u = d.id[i];
  const int c = d.nbr_cnt[i];
  cnt_out[u] = c;
  const int m = min(min(c, d.W), width);
  for (int s = 0; s < m; ++s) nbr_out[(size_t)u * width + s] = d.id[d.nbr[(size_t)s * d.N + i]];
}

__global__ void k_energy_out(Dev d, double* e, double* w) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= d.nbox) return;
  const int par = (int)(d.g->step & 1ull);
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
