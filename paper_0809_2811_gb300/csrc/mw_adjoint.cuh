// mw_adjoint.cuh -- adjoint of the forces for force-matching fits.
//
// The paper fits lambda, epsilon and sigma by scans (Sec. II.D); this is the
// gradient-based counterpart.  Given w = dL/dF (one vector per atom) let
//   D(x, theta) = sum_i w_i . grad_i E.
// Because F = -grad E:
//   dL/dx       = -grad_x D = -H w                (H = Hessian of E)
//   dL/depsilon = -D / epsilon                     (E is linear in epsilon)
//   dL/dlambda  = -D3 / lambda                     (E3 is linear in lambda)
//   dL/dsigma   = (D + sum_terms sum_legs r_leg . dD_term/dr_leg) / sigma
// the last from the reduced form E = epsilon E~(x / sigma) of Sec. II.A.
// Each term of E depends on its leg vectors r (centre -> partner); D_term =
// sum_legs dw_leg . dterm/dr_leg with dw = w_partner - w_centre, and
// dD_term/dr_leg is the forward-mode tangent of dterm/dr_leg along dw
// (H_term dw).  The leg and triplet quantities are recomputed here from the
// positions and the current neighbour list, never stored between calls.
//
// Layout mirrors k_force: kG lanes per centre find its legs (pair term done
// by the owner), a padded shared-memory table holds per leg u, ee, tr, nde,
// t = 1/(r - a sig), j and the tangents du = (dw - (u.dw) u)/r, rdot = u.dw;
// the (centre, leg j) items of a warp are spread over its lanes and each runs
// over the partner legs k of its centre.
#pragma once

#include "mw_device.cuh"

namespace mw {

struct AdjTable {
  float4 ue[kFAtoms * kLPad];   // ux, uy, uz, ee
  float4 aux[kFAtoms * kLPad];  // tr, nde, t, j (int bits)
  float4 du[kFAtoms * kLPad];   // du/dt along dw (x, y, z), rdot
  float gi[kFAtoms][4];         // three-body part of dL/dx on the centre
  int nl[kFAtoms];
};

struct AdjDev {
  const float4* w;   // dL/dF in sorted order
  float4* gx;        // dL/dx accumulator, sorted order
  double* acc;       // per box: D2, D3, RH
};

// Pair term phi2 and its first two r-derivatives (FP32).
__device__ __forceinline__ void phi2_d12(const FParams& P, float r, float invr, float t, float& d1, float& d2) {
  const float sr = P.sig * invr;
  float srp, srq;
  if (P.p == 4 && P.q == 0) {
    const float sr2 = sr * sr;
    srp = sr2 * sr2;
    srq = 1.0f;
  } else {
    srp = powi(sr, P.p);
    srq = powi(sr, P.q);
  }
  const float f = fmaf(P.B, srp, -srq);
  const float f1 = ((float)(-P.p) * P.B * srp + (float)P.q * srq) * invr;
  const float f2 = ((float)(P.p * (P.p + 1)) * P.B * srp - (float)(P.q * (P.q + 1)) * srq) * invr * invr;
  const float e = exp2f(P.sig_l2e * t);
  const float e1 = -P.sig * t * t * e;
  const float e2 = P.sig * t * t * t * e * (2.0f + P.sig * t);
  d1 = P.Aeps * (f1 * e + f * e1);
  d2 = P.Aeps * (f2 * e + 2.0f * f1 * e1 + f * e2);
}

__device__ void adjoint_block(const Dev& d, const AdjDev& A, const FParams& P, AdjTable& T, int blk) {
  const int lane = threadIdx.x & 31;
  const int g = threadIdx.x & (kG - 1);
  const int a = threadIdx.x / kG;
  const int i = blk * kFAtoms + a;
  const bool valid = i < d.N;
  float acc[3] = {0.f, 0.f, 0.f};  // D2, D3, RH
  float px = 0.f, py = 0.f, pz = 0.f;  // pair part of dL/dx_i
  uint4 qi = make_uint4(0u, 0u, 0u, 0u);
  float4 wi = make_float4(0.f, 0.f, 0.f, 0.f);
  int cnt = 0, b = -1;
  float L0 = 0.f, L1 = 0.f, L2 = 0.f;
  if (valid) {
    qi = d.q[i];
    b = (int)qi.w;
    wi = A.w[i];
    cnt = min(d.nbr_cnt[i], d.W);
    const Box& bx = d.box[b];
    L0 = bx.Lq[0];
    L1 = bx.Lq[1];
    L2 = bx.Lq[2];
  }
  T.gi[a][g] = 0.f;
  const int iters = __reduce_max_sync(kFull, (cnt + kG - 1) / kG);
  const unsigned gsh = lane & ~(kG - 1);
  const int* row = d.nbr + (size_t)(valid ? i : 0) * d.W;
  int nl = 0;
  for (int t = 0; t < iters; ++t) {
    const int s = g + kG * t;
    bool leg = false;
    float dx = 0.f, dy = 0.f, dz = 0.f, r2 = 1.f;
    int j = 0;
    if (s < cnt) {
      j = row[s];
      const uint4 qj = d.q[j];
      dx = fix_diff(qi.x, qj.x, L0);
      dy = fix_diff(qi.y, qj.y, L1);
      dz = fix_diff(qi.z, qj.z, L2);
      r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
      leg = r2 < P.rc2;
    }
    float4 ue = make_float4(0.f, 0.f, 0.f, 0.f), ax = ue, du = ue;
    if (leg) {
      const float invr = rsqrtf(r2);
      const float r = r2 * invr;
      leg = r < P.rc;
      if (leg) {
        const float ux = dx * invr, uy = dy * invr, uz = dz * invr;
        const float tinv = __fdividef(1.0f, r - P.rc);
        const float4 wj = A.w[j];
        const float wx = wj.x - wi.x, wy = wj.y - wi.y, wz = wj.z - wi.z;
        const float rd = fmaf(ux, wx, fmaf(uy, wy, uz * wz));
        const float dux = (wx - rd * ux) * invr, duy = (wy - rd * uy) * invr, duz = (wz - rd * uz) * invr;
        float d1, d2;
        phi2_d12(P, r, invr, tinv, d1, d2);
        // pair: dD/dr = phi'' rdot u + phi' du ; dL/dx_i = +dD/dr (owner)
        px = fmaf(d2 * rd, ux, fmaf(d1, dux, px));
        py = fmaf(d2 * rd, uy, fmaf(d1, duy, py));
        pz = fmaf(d2 * rd, uz, fmaf(d1, duz, pz));
        acc[0] = fmaf(0.5f * d1, rd, acc[0]);
        acc[2] = fmaf(0.5f * r * d2, rd, acc[2]);
        ue = make_float4(ux, uy, uz, P.sle * exp2f(P.gsig_l2e * tinv));
        ax = make_float4(2.0f * invr, P.gsig * tinv * tinv, tinv, __int_as_float(j));
        du = make_float4(dux, duy, duz, rd);
      }
    }
    const unsigned m = (__ballot_sync(kFull, leg) >> gsh) & ((1u << kG) - 1u);
    const int pos = nl + __popc(m & ((1u << g) - 1u));
    if (leg && pos < kLMax) {
      T.ue[a * kLPad + pos] = ue;
      T.aux[a * kLPad + pos] = ax;
      T.du[a * kLPad + pos] = du;
    }
    nl += __popc(m);
  }
  if (g == 0) T.nl[a] = valid ? nl : 0;
  __syncwarp();
  const int a0 = (threadIdx.x >> 5) * kWAtoms;
  int pre[kWAtoms + 1];
  pre[0] = 0;
#pragma unroll
  for (int k = 0; k < kWAtoms; ++k) {
    int n = T.nl[a0 + k];
    if (n > kLMax) n = 0;
    pre[k + 1] = pre[k] + n;
  }
  const int b0 = __shfl_sync(kFull, b, 0);
  const bool wuni = __all_sync(kFull, b == b0 || b < 0);
  const float c0 = P.c0;
  for (int base = 0; base < pre[kWAtoms]; base += 32) {
    const int it = base + lane;
    int ka = -1, first = 0, n = 0;
#pragma unroll
    for (int k = 0; k < kWAtoms; ++k)
      if (it >= pre[k] && it < pre[k + 1]) {
        ka = k;
        first = pre[k];
        n = pre[k + 1] - pre[k];
      }
    float hx = 0.f, hy = 0.f, hz = 0.f;  // sum over partners of d(dterm/dr_j)/dt
    if (ka >= 0) {
      const int aa = a0 + ka;
      const int jj = it - first;
      const int rb = aa * kLPad;
      const float4 uj = T.ue[rb + jj], xj = T.aux[rb + jj], vj = T.du[rb + jj];
      const float trj = xj.x, ndej = xj.y, tj = xj.z;
      const float rdj = vj.w;
      const float trdot = -0.5f * trj * trj * rdj;
      const float ndedot = -2.0f * ndej * tj * rdj;
      float Gx = 0.f, Gy = 0.f, Gz = 0.f;
      for (int k = 0; k < n; ++k) {
        if (k == jj) continue;
        const float4 uk = T.ue[rb + k];
        const float ndek = T.aux[rb + k].y;
        const float4 vk = T.du[rb + k];
        const float c = fmaf(uj.x, uk.x, fmaf(uj.y, uk.y, uj.z * uk.z));
        const float cd = fmaf(vj.x, uk.x, fmaf(vj.y, uk.y, fmaf(vj.z, uk.z,
                         fmaf(uj.x, vk.x, fmaf(uj.y, vk.y, uj.z * vk.z)))));
        const float D = c - c0;
        const float pk = uj.w * uk.w;
        const float gg = pk * D;
        const float gd = fmaf(-gg, fmaf(ndej, rdj, ndek * vk.w), pk * cd);
        const float av = gg * trj;
        const float ad = fmaf(gd, trj, gg * trdot);
        const float qv = fmaf(c, trj, D * ndej);
        const float qd = fmaf(cd, trj + ndej, fmaf(c, trdot, D * ndedot));
        const float bv = gg * qv;
        const float bd = fmaf(gd, qv, gg * qd);
        Gx = fmaf(av, uk.x, fmaf(-bv, uj.x, Gx));
        Gy = fmaf(av, uk.y, fmaf(-bv, uj.y, Gy));
        Gz = fmaf(av, uk.z, fmaf(-bv, uj.z, Gz));
        hx = fmaf(ad, uk.x, fmaf(av, vk.x, fmaf(-bd, uj.x, fmaf(-bv, vj.x, hx))));
        hy = fmaf(ad, uk.y, fmaf(av, vk.y, fmaf(-bd, uj.y, fmaf(-bv, vj.y, hy))));
        hz = fmaf(ad, uk.z, fmaf(av, vk.z, fmaf(-bd, uj.z, fmaf(-bv, vj.z, hz))));
      }
      // dw_j = r du_j + rdot u_j ;  r_j = 2 / tr_j
      const float rj = __fdividef(2.0f, trj);
      const float wx = fmaf(rj, vj.x, rdj * uj.x), wy = fmaf(rj, vj.y, rdj * uj.y), wz = fmaf(rj, vj.z, rdj * uj.z);
      const float d3 = fmaf(wx, Gx, fmaf(wy, Gy, wz * Gz));
      const float rh = rj * fmaf(uj.x, hx, fmaf(uj.y, hy, uj.z * hz));
      red_add_v4(A.gx + __float_as_int(xj.w), -hx, -hy, -hz);
      if (wuni) {
        acc[1] += d3;
        acc[2] += rh;
      } else {
        double* p = &A.acc[3 * d.q[blk * kFAtoms + aa].w];
        atomicAdd(p + 1, (double)d3);
        atomicAdd(p + 2, (double)rh);
      }
    }
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int ko = __shfl_up_sync(kFull, ka, o);
      const float tx = __shfl_up_sync(kFull, hx, o), ty = __shfl_up_sync(kFull, hy, o),
                  tz = __shfl_up_sync(kFull, hz, o);
      if (lane >= o && ko == ka) {
        hx += tx;
        hy += ty;
        hz += tz;
      }
    }
    const int kn = __shfl_down_sync(kFull, ka, 1);
    if (ka >= 0 && (lane == 31 || kn != ka)) {
      T.gi[a0 + ka][0] += hx;
      T.gi[a0 + ka][1] += hy;
      T.gi[a0 + ka][2] += hz;
    }
    __syncwarp();
  }
  __syncwarp();
#pragma unroll
  for (int o = 1; o < kG; o <<= 1) {
    px += __shfl_xor_sync(kFull, px, o);
    py += __shfl_xor_sync(kFull, py, o);
    pz += __shfl_xor_sync(kFull, pz, o);
  }
  if (valid && g == 0) {
    red_add_v4(A.gx + i, px + T.gi[a][0], py + T.gi[a][1], pz + T.gi[a][2]);
    if (nl > kLMax) {
      const int slot = atomicAdd(&d.g->n_over, 1);
      if (slot < d.N) d.over[slot] = i;
    }
  }
  const int ab = wuni ? b0 : b;
  box_accumulate<3>(acc, ab, [&](int bb) { return &A.acc[3 * bb]; });
}

__global__ void __launch_bounds__(kFThreads) k_adjoint(Dev d, AdjDev A, FParams P) {
  if (block_stop(d)) return;
  extern __shared__ __align__(16) unsigned char adj_smem[];
  AdjTable& T = *reinterpret_cast<AdjTable*>(adj_smem);
  adjoint_block(d, A, P, T, blockIdx.x);
}

// Three-body adjoint of centres with more than kLMax legs (rare): legs in
// local memory, ordered leg pairs, same arithmetic.
__device__ void adjoint_overflow_item(const Dev& d, const AdjDev& A, const FParams& P, int i) {
  const uint4 qi = d.q[i];
  const int b = (int)qi.w;
  const Box& bx = d.box[b];
  const float4 wi = A.w[i];
  int cnt = d.nbr_cnt[i];
  if (cnt > d.W) cnt = d.W;
  float4 U[kMaxLegsOverflow], X[kMaxLegsOverflow], V[kMaxLegsOverflow];
  int nl = 0;
  for (int s = 0; s < cnt; ++s) {
    const int j = d.nbr[(size_t)i * d.W + s];
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
    const float ux = dx * invr, uy = dy * invr, uz = dz * invr;
    const float tinv = __fdividef(1.0f, r - P.rc);
    const float4 wj = A.w[j];
    const float wx = wj.x - wi.x, wy = wj.y - wi.y, wz = wj.z - wi.z;
    const float rd = fmaf(ux, wx, fmaf(uy, wy, uz * wz));
    U[nl] = make_float4(ux, uy, uz, P.sle * exp2f(P.gsig_l2e * tinv));
    X[nl] = make_float4(2.0f * invr, P.gsig * tinv * tinv, tinv, __int_as_float(j));
    V[nl] = make_float4((wx - rd * ux) * invr, (wy - rd * uy) * invr, (wz - rd * uz) * invr, rd);
    ++nl;
  }
  float d3s = 0.f, rhs = 0.f, cx = 0.f, cy = 0.f, cz = 0.f;
  for (int jj = 0; jj < nl; ++jj) {
    const float4 uj = U[jj], xj = X[jj], vj = V[jj];
    const float trj = xj.x, ndej = xj.y, tj = xj.z, rdj = vj.w;
    const float trdot = -0.5f * trj * trj * rdj;
    const float ndedot = -2.0f * ndej * tj * rdj;
    float Gx = 0.f, Gy = 0.f, Gz = 0.f, hx = 0.f, hy = 0.f, hz = 0.f;
    for (int k = 0; k < nl; ++k) {
      if (k == jj) continue;
      const float4 uk = U[k], vk = V[k];
      const float ndek = X[k].y;
      const float c = fmaf(uj.x, uk.x, fmaf(uj.y, uk.y, uj.z * uk.z));
      const float cd = fmaf(vj.x, uk.x, fmaf(vj.y, uk.y, fmaf(vj.z, uk.z,
                       fmaf(uj.x, vk.x, fmaf(uj.y, vk.y, uj.z * vk.z)))));
      const float D = c - P.c0;
      const float pk = uj.w * uk.w;
      const float gg = pk * D;
      const float gd = fmaf(-gg, fmaf(ndej, rdj, ndek * vk.w), pk * cd);
      const float av = gg * trj;
      const float ad = fmaf(gd, trj, gg * trdot);
      const float qv = fmaf(c, trj, D * ndej);
      const float qd = fmaf(cd, trj + ndej, fmaf(c, trdot, D * ndedot));
      const float bv = gg * qv;
      const float bd = fmaf(gd, qv, gg * qd);
      Gx = fmaf(av, uk.x, fmaf(-bv, uj.x, Gx));
      Gy = fmaf(av, uk.y, fmaf(-bv, uj.y, Gy));
      Gz = fmaf(av, uk.z, fmaf(-bv, uj.z, Gz));
      hx = fmaf(ad, uk.x, fmaf(av, vk.x, fmaf(-bd, uj.x, fmaf(-bv, vj.x, hx))));
      hy = fmaf(ad, uk.y, fmaf(av, vk.y, fmaf(-bd, uj.y, fmaf(-bv, vj.y, hy))));
      hz = fmaf(ad, uk.z, fmaf(av, vk.z, fmaf(-bd, uj.z, fmaf(-bv, vj.z, hz))));
    }
    const float rj = __fdividef(2.0f, trj);
    const float wx = fmaf(rj, vj.x, rdj * uj.x), wy = fmaf(rj, vj.y, rdj * uj.y), wz = fmaf(rj, vj.z, rdj * uj.z);
    d3s = fmaf(wx, Gx, fmaf(wy, Gy, fmaf(wz, Gz, d3s)));
    rhs = fmaf(rj, fmaf(uj.x, hx, fmaf(uj.y, hy, uj.z * hz)), rhs);
    red_add_v4(A.gx + __float_as_int(xj.w), -hx, -hy, -hz);
    cx += hx;
    cy += hy;
    cz += hz;
  }
  red_add_v4(A.gx + i, cx, cy, cz);
  atomicAdd(&A.acc[3 * b + 1], (double)d3s);
  atomicAdd(&A.acc[3 * b + 2], (double)rhs);
}

__global__ void __launch_bounds__(128) k_adjoint_overflow(Dev d, AdjDev A, FParams P) {
  if (d.g->status) return;
  const int nover = min(d.g->n_over, d.N);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nover; k += gridDim.x * blockDim.x)
    adjoint_overflow_item(d, A, P, d.over[k]);
}

// dL/dF (caller's order, floats) -> sorted float4; clear outputs and counters.
__global__ void k_adj_prep(Dev d, AdjDev A, const float* __restrict__ w_user) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) d.g->n_over = 0;
  if (i < 3 * d.nbox) A.acc[i] = 0.0;
  if (i >= d.N) return;
  const int u = d.id[i];
  ((float4*)A.w)[i] = make_float4(w_user[3 * (size_t)u], w_user[3 * (size_t)u + 1], w_user[3 * (size_t)u + 2], 0.f);
  A.gx[i] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// dL/dx sorted -> caller's order.
__global__ void k_adj_out(Dev d, AdjDev A, float* __restrict__ g_user) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.N) return;
  const int u = d.id[i];
  const float4 v = A.gx[i];
  g_user[3 * (size_t)u] = v.x;
  g_user[3 * (size_t)u + 1] = v.y;
  g_user[3 * (size_t)u + 2] = v.z;
}

}  // namespace mw
