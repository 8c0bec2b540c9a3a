// mw_species.cuh -- energy, forces and virial of boxes holding several
// species (the paper's mW with solutes of their own lambda, epsilon, sigma,
// Sec. IV, and the SW family of Fig. 2 mixed): the Sec. II.A equations with
// a parameter set per ordered species triple.  The pair (i, j) takes the set
// of (ti, tj, tj); the three-body term of centre i with legs j, k takes
// lambda epsilon and cos theta0 of (ti, tj, tk) and each leg's exponential
// factor from that leg's pair set.  lambda epsilon then varies per leg pair,
// so the per-centre moment form of k_force applies only when it factors into
// leg weights, lambda epsilon of (a; b, c) = h_ab h_ac with cos theta0 set by
// the centre (geometric-mean mixing; a solute with lambda = 0): k_force_sp.
// Other tables keep the lane-group structure and walk the leg pairs of each
// centre in phase C (k_force_sp<., 2>).  Centres with more legs than the
// group stages go to species_item, one thread walking every leg pair with
// its legs in local memory, with the same pair-term ownership, scatter of
// the leg forces and per-box reductions.
#pragma once

#include "mw_device.cuh"

namespace mw {


// Owner contribution of centre i: pair terms (half energy, the whole force
// on the centre, half virial; the partner does the same from its side) and
// its three-body terms (every unordered leg pair once; the leg forces are
// scattered, the reaction stays with the centre).  Returns the centre's box.
template <bool kCount>
__device__ int species_item(const Dev& d, const SpPair* sp, const float2* st, int nsp, int i, float (&acc)[8]) {
  const uint4 qi = d.q[i];
  const int b = (int)qi.w;
  const Box& bx = d.box[b];
  const int ti = d.typ[i];
  const SpPair* spi = sp + ti * nsp;
  const float2* sti = st + ti * nsp * nsp;
  int cnt = d.nbr_cnt[i];
  if (cnt > d.W) cnt = d.W;
  float ux[kMaxLegsOverflow], uy[kMaxLegsOverflow], uz[kMaxLegsOverflow], tr[kMaxLegsOverflow],
      nde[kMaxLegsOverflow], ee[kMaxLegsOverflow], rr[kMaxLegsOverflow];
  float ax[kMaxLegsOverflow], ay[kMaxLegsOverflow], az[kMaxLegsOverflow];
  int jj[kMaxLegsOverflow], tt[kMaxLegsOverflow];
  int nl = 0;
  float px = 0.f, py = 0.f, pz = 0.f;
  for (int s = 0; s < cnt; ++s) {
    const int j = d.nbr[(size_t)i * d.W + s];
    const uint4 qj = d.q[j];
    const int tj = d.typ[j];
    const SpPair pp = spi[tj];
    const float dx = fix_diff(qi.x, qj.x, bx.Lq[0]), dy = fix_diff(qi.y, qj.y, bx.Lq[1]),
                dz = fix_diff(qi.z, qj.z, bx.Lq[2]);
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    if (r2 >= pp.rc2) continue;
    LegTerms lt;
    if (!leg_terms(r2, pp, lt)) continue;
    if (nl >= kMaxLegsOverflow) {
      set_status(d.g, ST_LEGS);
      d.g->err_index = i;
      break;
    }
    const float invr = lt.invr, r = lt.r;
    ux[nl] = dx * invr;
    uy[nl] = dy * invr;
    uz[nl] = dz * invr;
    tr[nl] = 2.0f * invr;
    nde[nl] = lt.nde;
    ee[nl] = lt.e3;
    rr[nl] = r;
    jj[nl] = j;
    tt[nl] = tj;
    ax[nl] = ay[nl] = az[nl] = 0.f;
    {  // pair term
      const float dphi = lt.dphi;
      acc[0] = fmaf(0.5f, lt.phi, acc[0]);
      px = fmaf(dphi, ux[nl], px);
      py = fmaf(dphi, uy[nl], py);
      pz = fmaf(dphi, uz[nl], pz);
      const float wv = -0.5f * dphi * r;
      acc[2] = fmaf(wv * ux[nl], ux[nl], acc[2]);
      acc[3] = fmaf(wv * uy[nl], uy[nl], acc[3]);
      acc[4] = fmaf(wv * uz[nl], uz[nl], acc[4]);
      acc[5] = fmaf(wv * ux[nl], uy[nl], acc[5]);
      acc[6] = fmaf(wv * ux[nl], uz[nl], acc[6]);
      acc[7] = fmaf(wv * uy[nl], uz[nl], acc[7]);
    }
    ++nl;
  }
  if (kCount) {
    atomicAdd((unsigned long long*)&d.g->npairs, (unsigned long long)nl);
    atomicAdd((unsigned long long*)&d.g->ntrip, (unsigned long long)(nl * (nl - 1) / 2));
  }
  for (int j = 0; j < nl; ++j) {
    const float2* stj = sti + tt[j] * nsp;
    for (int k = j + 1; k < nl; ++k) {
      const float2 lc = stj[tt[k]];  // (lambda epsilon, cos theta0) of (ti; tj, tk)
      const float c = fmaf(ux[j], ux[k], fmaf(uy[j], uy[k], uz[j] * uz[k]));
      const float D = c - lc.y;
      const float g = lc.x * ee[j] * ee[k] * D;
      acc[1] = fmaf(g, D, acc[1]);
      const float aj = g * tr[j], bj = g * fmaf(c, tr[j], D * nde[j]);
      ax[j] = fmaf(-aj, ux[k], fmaf(bj, ux[j], ax[j]));
      ay[j] = fmaf(-aj, uy[k], fmaf(bj, uy[j], ay[j]));
      az[j] = fmaf(-aj, uz[k], fmaf(bj, uz[j], az[j]));
      const float ak = g * tr[k], bk = g * fmaf(c, tr[k], D * nde[k]);
      ax[k] = fmaf(-ak, ux[j], fmaf(bk, ux[k], ax[k]));
      ay[k] = fmaf(-ak, uy[j], fmaf(bk, uy[k], ay[k]));
      az[k] = fmaf(-ak, uz[j], fmaf(bk, uz[k], az[k]));
    }
  }
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
  red_add_v4(d.f + i, fx + px, fy + py, fz + pz);
  return b;
}

// Force phase of a box set holding several species: the lane-group kernel
// with per-leg constants, kMode 1 (tables whose three-body strengths factor
// into leg weights, lambda epsilon of (a; b, c) = h_ab h_ac with cos theta0
// of the centre: the moment form) or kMode 2 (any table: leg pairs walked
// in phase C).  P.rc is the widest pair cutoff.  Block 0 consumes the
// rebuild flags.
template <bool kCount, int kMode>
__global__ void __launch_bounds__(kFThreads, 4) k_force_sp(const __grid_constant__ Dev d, const __grid_constant__ FParams P) {
  if (block_stop(d)) return;
  __shared__ LegTableSp T;
  __shared__ SpPair sp[kMaxSpecies * kMaxSpecies];
  __shared__ float2 st[kMode == 2 ? kMaxSpecies * kMaxSpecies * kMaxSpecies : 1];
  const int nsp = d.nsp;
  for (int k = threadIdx.x; k < nsp * nsp; k += blockDim.x) sp[k] = d.sp_pair[k];
  if constexpr (kMode == 2)
    for (int k = threadIdx.x; k < nsp * nsp * nsp; k += blockDim.x) st[k] = d.sp_tri[k];
  const int par = (int)(d.g->step & 1ull);
  if (blockIdx.x == 0) {
    for (int k = threadIdx.x; k < d.nbox; k += blockDim.x) d.bst[k].rebuild = 0;
    if (threadIdx.x == 0) {
      d.g->any_rebuild = 0;
      d.g->wpar = par;
    }
  }
  __syncthreads();
  force_block<kCount, kMode>(d, P, T, blockIdx.x, par, sp, nsp, st);
}

// Sorted species from the caller-order ones (after a new state or a new
// species assignment; the sorts carry them from then on).
__global__ void k_gather_types(Dev d) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < d.N) d.typ[i] = d.utyp[d.id[i]];
}

}  // namespace mw
